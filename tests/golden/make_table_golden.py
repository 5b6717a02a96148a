"""Writes tests/golden/gb300_full_f17_times.txt from a timing table that
``bench.py --table-out PATH`` recorded (JSON lines, one row per configuration).

The golden file keeps, per measured configuration of the full space, its
canonical index and median time; a header names the command, device, kernel
source and clock it came from.  It is measured data (a timing landscape), not
a computed result: the strategy tests replay it and compare each strategy's
pick with the exhaustive optimum that oracle.analysis ranks from the same file.

    python tests/golden/make_table_golden.py TABLE.jsonl --device "NVIDIA GB300" \
        --kernel-sha e49de8f102ae6b61 --command "python bench.py ..." --clock "2070 MHz"
"""
import argparse
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "gb300_full_f17_times.txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("table")
    ap.add_argument("--device", required=True)
    ap.add_argument("--kernel-sha", required=True)
    ap.add_argument("--command", required=True)
    ap.add_argument("--clock", required=True)
    ap.add_argument("--date", required=True)
    a = ap.parse_args()
    rows = [json.loads(line) for line in open(a.table)]
    problems = {r["problem"] for r in rows}
    assert len(problems) == 1, problems
    with open(OUT, "w") as fh:
        fh.write("# Brute-force timing table of the full space (5,576 valid configurations), one GB300.\n")
        fh.write(f"# problem: {problems.pop()} (output 4096x4096, filter 17x17, uniform[-1,1) seed 1)\n")
        fh.write(f"# command: {a.command}\n")
        fh.write(f"# device: {a.device}; SM clock during the run: {a.clock}; date: {a.date}\n")
        fh.write(f"# kernel source: corr2d.cuh sha256[:16] = {a.kernel_sha}\n")
        fh.write("# per row: canonical index (full space, Table-1 order), median of 7 event-timed launches in ms"
                 " (nan: failed)\n")
        for r in sorted(rows, key=lambda r: r["index"]):
            t = r["t_med_ms"]
            ok = r["status"] == 0 and t is not None and math.isfinite(t)
            fh.write(f"{r['index']} {t!r}\n" if ok else f"{r['index']} nan\n")
    print(OUT, len(rows))


if __name__ == "__main__":
    main()
