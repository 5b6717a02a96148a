"""GPU tests of the continuous-batching server: every result matches the FP64
oracle and the single-problem kernel bit for bit, a request gives the same
bits alone and in a mix of concurrent requests, resident images work, the
memory budget bounds admission, and the host-side waits and errors behave."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


def _req(seed, side, fs):
    img, f = synthetic.make_problem(seed, side, side, fs, fs)
    h_img = torch.from_numpy(img).pin_memory()
    h_out = torch.full((side, synthetic.round_up(side, 4)), float("nan")).pin_memory()
    return img, np.ascontiguousarray(f), h_img, h_out


def _single(ct, img, f, side, fs, device):
    d = torch.from_numpy(img).to(device)
    out = ct.conv2d(d, f, ct.config(32, 4, 4, 2, 1, 1), in_w=side + fs - 1)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def server(ctlib, cuda_device):
    s = ctlib.Server(1 << 30, tune=False, max_batch=16, max_launches=3, max_wait_us=100)
    yield s
    s.close()


def test_alone_and_in_the_mix(ctlib, cuda_device, server):
    target = _req(900, 333, 11)
    img, f, h_img, h_out = target
    rid = server.submit(h_out, f, 333, 333, h_image=h_img)
    server.wait(rid, 10_000_000)
    alone = h_out.numpy()[:, :333].copy()
    ref, S = oracle.corr2d_f64(img, f, 333, 333)
    assert_parity(alone, ref, S, "served alone")
    assert np.array_equal(alone.view(np.uint32), _single(ctlib, img, f, 333, 11, cuda_device).view(np.uint32))

    # the same request submitted in the middle of 40 others of mixed sizes
    shapes = synthetic.uneven_batch(31, 40, 64, 900, (3, 5, 7, 9, 11, 13, 15, 17))
    reqs = [_req(1000 + k, side, fs) for k, (side, fs) in enumerate(shapes)]
    target2 = _req(900, 333, 11)
    ids = []
    for k, ((im, ff, hi, ho), (side, fs)) in enumerate(zip(reqs, shapes)):
        ids.append(server.submit(ho, ff, side, side, h_image=hi))
        if k == 20:
            tid = server.submit(target2[3], target2[1], 333, 333, h_image=target2[2])
    for rid in ids:
        server.wait(rid, 30_000_000)
    server.wait(tid, 30_000_000)
    assert np.array_equal(target2[3].numpy()[:, :333].view(np.uint32), alone.view(np.uint32))
    for (im, ff, hi, ho), (side, fs) in zip(reqs, shapes):
        got = ho.numpy()[:, :side]
        assert np.array_equal(got.view(np.uint32), _single(ctlib, im, ff, side, fs, cuda_device).view(np.uint32))
    st = server.stats()
    assert st["completed"] >= 42 and st["failed"] == 0
    assert st["launches"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0


def test_resident_image(ctlib, cuda_device, server):
    side, fmax = 400, 17
    img, _ = synthetic.make_problem(77, side, side, fmax, fmax)
    h_img = torch.from_numpy(img).pin_memory()
    iid = server.register_image(h_img, in_w=side + fmax - 1)
    outs = []
    for k, fs in enumerate((3, 9, 17)):
        f = synthetic.uniform_pm1(500 + k, 0, fs * fs).reshape(fs, fs)
        ow = side + fmax - fs          # the largest output the resident image allows
        h_out = torch.empty((ow, synthetic.round_up(ow, 4))).pin_memory()
        outs.append((server.submit(h_out, f, ow, ow, image_id=iid), h_out, f, ow))
    for rid, h_out, f, ow in outs:
        server.wait(rid, 10_000_000)
        ref, S = oracle.corr2d_f64(img, f, ow, ow)
        assert_parity(h_out.numpy()[:, :ow], ref, S, "resident image")
    server.release_image(iid)


def test_budget_admission(ctlib, cuda_device):
    # about 2.3 MB per request (image + output) against a 6 MB budget: at
    # most two requests are resident at once, all complete
    s = ctlib.Server(6 << 20, tune=False, max_batch=8, staging_bytes=1 << 20)
    try:
        reqs = [_req(3000 + k, 500, 5) for k in range(10)]
        ids = [s.submit(ho, f, 500, 500, h_image=hi) for (_, f, hi, ho) in reqs]
        for rid in ids:
            s.wait(rid, 30_000_000)
        st = s.stats()
        assert st["completed"] == 10 and st["peak_mem_bytes"] <= 6 << 20
        for (img, f, hi, ho) in reqs[:3]:
            ref, S = oracle.corr2d_f64(img, f, 500, 500)
            assert_parity(ho.numpy()[:, :500], ref, S, "budgeted")
        # a request larger than the whole budget is refused at submit
        big = _req(3100, 1500, 5)
        with pytest.raises(ctlib.CTError) as e:
            s.submit(big[3], big[1], 1500, 1500, h_image=big[2])
        assert e.value.status == -6
    finally:
        s.close()


def test_wait_timeout_and_unsupported_filter(ctlib, cuda_device, server):
    img, f, h_img, h_out = _req(4000, 2048, 17)
    rid = server.submit(h_out, f, 2048, 2048, h_image=h_img)
    with pytest.raises(ctlib.CTError) as e:
        server.wait(rid, 0)
    assert e.value.status == -7
    server.wait(rid, 30_000_000)              # still collectable after the timeout
    assert np.isfinite(h_out.numpy()[:, :2048]).all()
    _, f4, hi4, ho4 = _req(4001, 64, 4)
    with pytest.raises(ctlib.CTError) as e:
        server.submit(ho4, f4, 64, 64, h_image=hi4)
    assert e.value.status == -8


def test_tuned_server(ctlib, cuda_device):
    s = ctlib.Server(1 << 30, tune=True, filter_min=3, filter_max=7)
    try:
        img, f, h_img, h_out = _req(5000, 700, 7)
        s.wait(s.submit(h_out, f, 700, 700, h_image=h_img), 30_000_000)
        ref, S = oracle.corr2d_f64(img, f, 700, 700)
        assert_parity(h_out.numpy()[:, :700], ref, S, "tuned server")
    finally:
        s.close()


@pytest.mark.parametrize("paced", [False, True], ids=["closed_loop", "poisson"])
def test_native_run_same_bits(ctlib, cuda_device, server, paced):
    """ct_server_run drives a stream from native threads (closed loop with at
    most 8 requests in flight, or paced by Poisson arrival times at 4,000/s):
    every request completes, each result is the single-problem kernel's bits,
    output buffers shared by requests 8 apart are safe, and the statistics
    cover the run (latencies, kernel busy time within the wall time)."""
    shapes = synthetic.uneven_batch(77, 48, 64, 700, (3, 5, 9, 17))
    K = 8
    reqs, outs, probs = [], [], []
    for k, (side, fs) in enumerate(shapes):
        img, f, h_img, _ = _req(2000 + k, side, fs)
        probs.append((img, f, side, fs))
    slots = [torch.full((700 * 700,), float("nan")).pin_memory() for _ in range(K)]
    results = {}
    # run the stream in chunks of K so every request's output can be read before its slot is reused
    lat_all = []
    for c0 in range(0, len(shapes), K):
        chunk = []
        for k in range(c0, min(len(shapes), c0 + K)):
            img, f, side, fs = probs[k]
            h_img = torch.from_numpy(img).pin_memory()
            h_out = slots[k % K][:side * synthetic.round_up(side, 4)].view(side, synthetic.round_up(side, 4))
            outs.append(h_img)
            chunk.append(server.request(h_out, f, side, side, h_image=h_img))
        arrivals = np.cumsum(np.full(len(chunk), 1.0 / 4000.0)) if paced else None
        st, lat = server.run(chunk, arrival_s=arrivals, max_in_flight=K)
        assert st["completed"] == len(chunk) and st["failed"] == 0
        assert np.all(np.isfinite(lat)) and np.all(lat > 0)
        assert 0.0 < st["kernel_busy_s"] <= st["wall_s"] * 1.05 and st["kernel_busy_frac"] <= 1.05
        lat_all += list(lat)
        for k in range(c0, min(len(shapes), c0 + K)):
            side = probs[k][2]
            results[k] = slots[k % K][:side * synthetic.round_up(side, 4)].view(side, -1).numpy()[:, :side].copy()
    for k, (img, f, side, fs) in enumerate(probs):
        assert np.array_equal(results[k].view(np.uint32), _single(ctlib, img, f, side, fs, cuda_device).view(np.uint32))
    assert len(lat_all) == len(shapes)
