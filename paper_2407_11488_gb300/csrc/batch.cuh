// Persistent batched correlation: one launch works through a list of tiles
// that belong to many problems of uneven image and filter sizes.
//
// Compiled at run time by NVRTC to an sm_103a cubin.  Every problem belongs to
// a bucket (same filter size, similar image size); each bucket has its own
// compile-time tile routine (filter size, block shape, register tile), chosen
// by the library's tuner, and one launch holds all of them.  Each block
// repeatedly takes the next work item (problem, tile) from a global counter.
// One thread stages an item with the Tensor Memory Accelerator: a 2D tensor
// copy of the tile's input halo (the box of the problem's tensor map; parts
// outside the image read as zero) and a bulk copy of the problem's filter
// taps, both completing on the buffer's mbarrier, into one of two
// shared-memory buffers while the block computes the previous item from the
// other.
//
// The per-output arithmetic is that of the single-problem kernel: one FP32
// fused multiply-add per tap, taps added in (i, j) order, so results are
// bit-identical to ct_corr2d for the same inputs.
//
// Macros: CT_NT (threads per block), CT_DTYPE (0 FP32, 1 BF16 image; BF16
// stays BF16 in shared memory and is widened when a row enters registers),
// CT_NB (buckets), and for every bucket b < CT_NB: CT_B<b>_BX (block width;
// block height = CT_NT / BX), CT_B<b>_TX, CT_B<b>_TY (register tile),
// CT_B<b>_UN (1: input-row loop unrolled), CT_B<b>_P2 (1, with UN = 1 and an
// even TY: paired multiply-adds, below), CT_B<b>_FW, CT_B<b>_FH (filter);
// CT_MINB (blocks per SM the register allocation must allow); CT_BUF_BYTES,
// the size of one item buffer (the largest bucket's, a multiple of 128).
//
// Filters are stored FP32, every filter starting on a 16-byte boundary: FH
// rows of taps, each padded with zeros to a multiple of 4, then (for the
// paired form) FH - 1 rows of tap pairs, row i - 1 holding (f[i][j],
// f[i-1][j]) for j < FW, padded with zero pairs to an even count.  Waits on
// an mbarrier give up after about two seconds: the block then sets bit 0 of
// counter[1], waits (again bounded) for the copies it started, and exits.

#ifndef CT_DTYPE
#define CT_DTYPE 0
#endif
// Test hook: bytes expected per item on top of those the copies deliver.  A
// nonzero value makes every wait run out, which exercises the bounded-wait
// path; it is 0 in every normal build.
#ifndef CT_TEST_EXTRA_TX
#define CT_TEST_EXTRA_TX 0
#endif

typedef long long ct_i64;
typedef unsigned int ct_u32;
typedef unsigned long long ct_u64;
#if CT_DTYPE == 0
typedef float ct_in_t;
#define CT_ESZ 4
#else
typedef unsigned short ct_in_t;
#define CT_ESZ 2
#endif
#define CT_BOXQ (16 / CT_ESZ)   // elements per 16 bytes; the halo box width is a multiple

struct CtBatchProblem {
    const ct_in_t* in;
    float* out;
    ct_i64 in_pitch, out_pitch;
    int out_w, out_h, in_w, in_h;
    int bucket, tiles_x, filt_off, pad;   // tiles_x: tile columns (for inspection; work items carry their tile)
};

struct CtBatchParams {
    const CtBatchProblem* probs;
    // per work item: (problem index, (tile row << 16) | tile column, bucket,
    // the problem's filt_off): all a block needs to stage and dispatch an
    // item, in one 16-byte load
    const uint4* work;
    const float* filters;         // all filters, FP32 (layout above), problem p at filt_off
    const unsigned char* tmaps;   // problem p's tensor map (128 bytes) at tmaps + 128 p
    unsigned int* counter;        // [0]: next work item, zero before the launch; [1]: error bits
    int n_work;
};

__device__ __forceinline__ constexpr int ct_rup(int v, int m) { return (v + m - 1) / m * m; }

// Two FP32 values in one 64-bit register pair, and the paired fused
// multiply-add: d = a * b + c in each half, each half an fma.rn.f32.
__device__ __forceinline__ ct_u64 ct_pk(float lo, float hi)
{
    ct_u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void ct_upk(ct_u64 r, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ ct_u64 ct_fma2(ct_u64 a, ct_u64 b, ct_u64 c)
{
    ct_u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ ct_u32 ct_sa(const void* p) { return (ct_u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ct_mbar_init(ct_u64* bar, ct_u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(ct_sa(bar)), "r"(count) : "memory");
}
// Makes the initialised barriers visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void ct_mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void ct_mbar_expect_tx(ct_u64* bar, ct_u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ct_sa(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool ct_mbar_try_wait(ct_u64* bar, ct_u32 parity)
{
    ct_u32 done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(ct_sa(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ ct_u64 ct_globaltimer()
{
    ct_u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Waits until the phase with the given parity of bar has completed; false
// after about two seconds without completion.
__device__ __forceinline__ bool ct_mbar_wait(ct_u64* bar, ct_u32 parity)
{
    if (ct_mbar_try_wait(bar, parity)) return true;
    const ct_u64 t0 = ct_globaltimer();
    while (!ct_mbar_try_wait(bar, parity))
        if (ct_globaltimer() - t0 > 2000000000ull) return false;
    return true;
}
// Orders the host's write of a tensor map before its use by the TMA unit.
__device__ __forceinline__ void ct_tmap_acquire(const void* tmap)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;\n" ::"l"(tmap) : "memory");
}
__device__ __forceinline__ void ct_tma_load_2d(void* dst, const void* tmap, int x, int y, ct_u64* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(ct_sa(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(ct_sa(bar))
        : "memory");
}
__device__ __forceinline__ void ct_bulk_load(void* dst, const void* src, ct_u32 bytes, ct_u64* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     ct_sa(dst)),
                 "l"(src), "r"(bytes), "r"(ct_sa(bar))
                 : "memory");
}

// Shared-memory buffer of one work item: the input tile plus halo (HH rows of
// SW elements, the tensor map's box, at offset 0), then the filter taps (FH
// rows of FWP floats, zero padded) at TAPS_OFF.  compute() is a real call, not
// inlined: each bucket's routine then gets its own register allocation and the
// kernel needs only the largest of them, instead of the union a single inlined
// body would hold.
template <int BX, int TX, int TY, int FW, int FH, int UN, int P2>
struct CtTile {
    static constexpr int BY = CT_NT / BX;
    static constexpr int TW = BX * TX, TH = BY * TY;
    static constexpr int HW = TW + FW - 1, HH = TH + FH - 1;
    static constexpr int SW = ct_rup(HW, CT_BOXQ);
    static constexpr int FWP = ct_rup(FW, 4);
    static constexpr int FWP2 = ct_rup(FW, 2);   // tap pairs per pair row
    static constexpr int HALO_BYTES = HH * SW * CT_ESZ;
    static constexpr int TAPS_OFF = ct_rup(HALO_BYTES, 16);
    static constexpr int PAIRS_OFF = FH * FWP * 4;   // from TAPS_OFF
    static constexpr int TAP_BYTES = PAIRS_OFF + (P2 ? (FH - 1) * FWP2 * 8 : 0);
    static_assert(!P2 || (UN == 1 && TY % 2 == 0), "the paired form needs an unrolled row loop and an even TY");
    static constexpr int VW = (TX % 4 == 0) ? 4 : ((TX % 2 == 0) ? 2 : 1);
    static constexpr int WW = TX + FW - 1;
    static constexpr int WWV = ct_rup(WW, VW);
    static_assert(SW <= 256 && HH <= 256, "the halo box exceeds 256 elements per side");
    static_assert(ct_rup(TAPS_OFF + TAP_BYTES, 128) <= CT_BUF_BYTES, "item buffer too small");
    static_assert(TW % 16 == 0, "tile columns must start on 16-element boundaries");

    // Thread 0: starts both copies of one item into buf, completing on bar.
    static __device__ __forceinline__ void stage(const unsigned char* tmap, const float* taps, ct_u32 tile,
                                                 unsigned char* buf, ct_u64* bar)
    {
        const int gx0 = (int)(tile & 0xffffu) * TW, gy0 = (int)(tile >> 16) * TH;
        ct_mbar_expect_tx(bar, (ct_u32)(HALO_BYTES + TAP_BYTES + CT_TEST_EXTRA_TX));
        ct_tma_load_2d(buf, tmap, gx0, gy0, bar);
        ct_bulk_load(buf + TAPS_OFF, taps, (ct_u32)TAP_BYTES, bar);
    }

    // Input row `row` of the thread's window, columns lx .. lx+WWV-1, as FP32.
    static __device__ __forceinline__ void load_window(const ct_in_t* halo, int row, int lx, float (&w)[WWV])
    {
        const ct_in_t* s = halo + row * SW + lx;
#pragma unroll
        for (int k = 0; k < WWV; k += VW) {
#if CT_DTYPE == 0
            if (VW == 4) {
                const float4 v = *reinterpret_cast<const float4*>(s + k);
                w[k] = v.x; w[k + 1] = v.y; w[k + 2] = v.z; w[k + 3] = v.w;
            } else if (VW == 2) {
                const float2 v = *reinterpret_cast<const float2*>(s + k);
                w[k] = v.x; w[k + 1] = v.y;
            } else {
                w[k] = s[k];
            }
#else
            if (VW == 4) {
                const uint2 v = *reinterpret_cast<const uint2*>(s + k);
                w[k] = __uint_as_float(v.x << 16); w[k + 1] = __uint_as_float(v.x & 0xffff0000u);
                w[k + 2] = __uint_as_float(v.y << 16); w[k + 3] = __uint_as_float(v.y & 0xffff0000u);
            } else if (VW == 2) {
                const ct_u32 v = *reinterpret_cast<const ct_u32*>(s + k);
                w[k] = __uint_as_float(v << 16); w[k + 1] = __uint_as_float(v & 0xffff0000u);
            } else {
                w[k] = __uint_as_float(((ct_u32)s[k]) << 16);
            }
#endif
        }
    }

    static __device__ __forceinline__ void row_step(const ct_in_t* halo, const float* taps, int lx, int ly, int r,
                                                    float (&acc)[TY][TX])
    {
        float w[WWV];
        load_window(halo, ly + r, lx, w);
#pragma unroll
        for (int ty = 0; ty < TY; ++ty) {
            const int i = r - ty;
            if (i >= 0 && i < FH) {
                float f[FWP];
#pragma unroll
                for (int q = 0; q < FWP; q += 4) {
                    const float4 t = *reinterpret_cast<const float4*>(taps + i * FWP + q);
                    f[q] = t.x; f[q + 1] = t.y; f[q + 2] = t.z; f[q + 3] = t.w;
                }
#pragma unroll
                for (int j = 0; j < FW; ++j)
#pragma unroll
                    for (int tx = 0; tx < TX; ++tx) acc[ty][tx] = fmaf(w[tx + j], f[j], acc[ty][tx]);
            }
        }
    }

    // Paired form: output rows 2k and 2k+1 of the thread's tile share each
    // input row r, with filter rows i = r - 2k and i - 1.  Where both exist,
    // one paired multiply-add per (pair, column, tap) does both, its taps a
    // (f[i][j], f[i-1][j]) pair from the pair rows (two pairs per 16-byte
    // broadcast load) and its input the window value in both halves; at the
    // two ends of a pair's input rows only one filter row exists (i = 0 for
    // row 2k, i = FH for row 2k+1: a scalar FMA on that half).  Each output
    // still adds its taps in (i, j) order, one fma.rn.f32 each.
    static __device__ __forceinline__ void row_step2(const ct_in_t* halo, const float* taps, int lx, int ly, int r,
                                                     ct_u64 (&acc2)[TY / 2][TX])
    {
        float w[WWV];
        load_window(halo, ly + r, lx, w);
        const float* pairs = taps + PAIRS_OFF / 4;
#pragma unroll
        for (int k = 0; k < TY / 2; ++k) {
            const int i = r - 2 * k;
            if (i >= 1 && i < FH) {
#pragma unroll
                for (int q = 0; q < FW; q += 2) {
                    const float4 t = *reinterpret_cast<const float4*>(pairs + ((i - 1) * FWP2 + q) * 2);
                    const ct_u64 f0 = ct_pk(t.x, t.y), f1 = ct_pk(t.z, t.w);
#pragma unroll
                    for (int tx = 0; tx < TX; ++tx) acc2[k][tx] = ct_fma2(ct_pk(w[tx + q], w[tx + q]), f0, acc2[k][tx]);
                    if (q + 1 < FW) {
#pragma unroll
                        for (int tx = 0; tx < TX; ++tx)
                            acc2[k][tx] = ct_fma2(ct_pk(w[tx + q + 1], w[tx + q + 1]), f1, acc2[k][tx]);
                    }
                }
            } else if (i == 0 || i == FH) {
                const int fi = i == 0 ? 0 : FH - 1;
#pragma unroll
                for (int q = 0; q < FW; q += 4) {
                    const float4 t = *reinterpret_cast<const float4*>(taps + fi * FWP + q);
                    const float f[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (q + e < FW) {
#pragma unroll
                            for (int tx = 0; tx < TX; ++tx) {
                                float lo, hi;
                                ct_upk(acc2[k][tx], lo, hi);
                                if (i == 0) lo = fmaf(w[tx + q + e], f[e], lo);
                                else hi = fmaf(w[tx + q + e], f[e], hi);
                                acc2[k][tx] = ct_pk(lo, hi);
                            }
                        }
                    }
                }
            }
        }
    }

    // Computes and stores one item whose halo and taps are in buf.
    static __device__ __noinline__ void compute(const CtBatchProblem& pr, ct_u32 tile, const unsigned char* buf)
    {
        const int tid = threadIdx.x;
        const ct_in_t* halo = reinterpret_cast<const ct_in_t*>(buf);
        const float* taps = reinterpret_cast<const float*>(buf + TAPS_OFF);
        const int gx0 = (int)(tile & 0xffffu) * TW, gy0 = (int)(tile >> 16) * TH;
        const int lx = (tid % BX) * TX, ly = (tid / BX) * TY;
        float acc[TY][TX];
#pragma unroll
        for (int ty = 0; ty < TY; ++ty)
#pragma unroll
            for (int tx = 0; tx < TX; ++tx) acc[ty][tx] = 0.0f;

        // Input rows slide through a register window once each; row r feeds
        // every output row ty with filter row i = r - ty, whose taps are read
        // as broadcast 16-byte loads.  UN = 1 unrolls the row loop (constant
        // offsets, no per-row predicates); UN = 0 keeps it rolled.  Per output
        // the taps are added in (i, j) order either way.
        if constexpr (P2 != 0) {
            ct_u64 acc2[TY / 2][TX];
#pragma unroll
            for (int k = 0; k < TY / 2; ++k)
#pragma unroll
                for (int tx = 0; tx < TX; ++tx) acc2[k][tx] = ct_pk(0.0f, 0.0f);
#pragma unroll
            for (int r = 0; r < TY + FH - 1; ++r) row_step2(halo, taps, lx, ly, r, acc2);
#pragma unroll
            for (int k = 0; k < TY / 2; ++k)
#pragma unroll
                for (int tx = 0; tx < TX; ++tx) ct_upk(acc2[k][tx], acc[2 * k][tx], acc[2 * k + 1][tx]);
        } else if constexpr (UN != 0) {
#pragma unroll
            for (int r = 0; r < TY + FH - 1; ++r) row_step(halo, taps, lx, ly, r, acc);
        } else {
#pragma unroll 1
            for (int r = 0; r < TY + FH - 1; ++r) row_step(halo, taps, lx, ly, r, acc);
        }

        const int gx = gx0 + lx, gy = gy0 + ly;
#pragma unroll
        for (int ty = 0; ty < TY; ++ty) {
            const int y = gy + ty;
            if (y < pr.out_h) {
                float* __restrict__ orow = pr.out + (ct_i64)y * pr.out_pitch + gx;
                if (TX % 4 == 0) {
#pragma unroll
                    for (int k = 0; k < TX; k += 4) {
                        if (gx + k + 3 < pr.out_w) {
                            *reinterpret_cast<float4*>(orow + k) =
                                make_float4(acc[ty][k], acc[ty][k + 1], acc[ty][k + 2], acc[ty][k + 3]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (gx + k + e < pr.out_w) orow[k + e] = acc[ty][k + e];
                        }
                    }
                } else {
#pragma unroll
                    for (int tx = 0; tx < TX; ++tx)
                        if (gx + tx < pr.out_w) orow[tx] = acc[ty][tx];
                }
            }
        }
    }
};

#define CT_TILE(b) \
    CtTile<CT_B##b##_BX, CT_B##b##_TX, CT_B##b##_TY, CT_B##b##_FW, CT_B##b##_FH, CT_B##b##_UN, CT_B##b##_P2>

// Thread 0: starts the copies of the work item `it` (its record) into buf.
// The tensor map, written by the host before the launch, is acquired for the
// tensor copies before this thread's first use of it; a block's items come
// in work-list order, so a problem's map is acquired again only when the
// thread's previous item belonged to another problem (*fenced).
__device__ __forceinline__ void ct_stage_item(const CtBatchParams& p, uint4 it, unsigned char* buf, ct_u64* bar,
                                              ct_u32* fenced)
{
    const unsigned char* tmap = p.tmaps + 128ull * it.x;
    if (*fenced != it.x) {
        ct_tmap_acquire(tmap);
        *fenced = it.x;
    }
    const float* taps = p.filters + it.w;
#define CT_STAGE_CASE(b) \
    case b: CT_TILE(b)::stage(tmap, taps, it.y, buf, bar); break;
    switch (it.z) {
#if CT_NB > 0
    CT_STAGE_CASE(0)
#endif
#if CT_NB > 1
    CT_STAGE_CASE(1)
#endif
#if CT_NB > 2
    CT_STAGE_CASE(2)
#endif
#if CT_NB > 3
    CT_STAGE_CASE(3)
#endif
#if CT_NB > 4
    CT_STAGE_CASE(4)
#endif
#if CT_NB > 5
    CT_STAGE_CASE(5)
#endif
#if CT_NB > 6
    CT_STAGE_CASE(6)
#endif
#if CT_NB > 7
    CT_STAGE_CASE(7)
#endif
#if CT_NB > 8
    CT_STAGE_CASE(8)
#endif
#if CT_NB > 9
    CT_STAGE_CASE(9)
#endif
#if CT_NB > 10
    CT_STAGE_CASE(10)
#endif
#if CT_NB > 11
    CT_STAGE_CASE(11)
#endif
#if CT_NB > 12
    CT_STAGE_CASE(12)
#endif
#if CT_NB > 13
    CT_STAGE_CASE(13)
#endif
#if CT_NB > 14
    CT_STAGE_CASE(14)
#endif
#if CT_NB > 15
    CT_STAGE_CASE(15)
#endif
    default: break;
    }
#undef CT_STAGE_CASE
}

__device__ __forceinline__ void ct_compute_item(const CtBatchProblem& pr, ct_u32 tile, ct_u32 bucket,
                                                const unsigned char* buf)
{
#define CT_COMPUTE_CASE(b) \
    case b: CT_TILE(b)::compute(pr, tile, buf); break;
    switch (bucket) {
#if CT_NB > 0
    CT_COMPUTE_CASE(0)
#endif
#if CT_NB > 1
    CT_COMPUTE_CASE(1)
#endif
#if CT_NB > 2
    CT_COMPUTE_CASE(2)
#endif
#if CT_NB > 3
    CT_COMPUTE_CASE(3)
#endif
#if CT_NB > 4
    CT_COMPUTE_CASE(4)
#endif
#if CT_NB > 5
    CT_COMPUTE_CASE(5)
#endif
#if CT_NB > 6
    CT_COMPUTE_CASE(6)
#endif
#if CT_NB > 7
    CT_COMPUTE_CASE(7)
#endif
#if CT_NB > 8
    CT_COMPUTE_CASE(8)
#endif
#if CT_NB > 9
    CT_COMPUTE_CASE(9)
#endif
#if CT_NB > 10
    CT_COMPUTE_CASE(10)
#endif
#if CT_NB > 11
    CT_COMPUTE_CASE(11)
#endif
#if CT_NB > 12
    CT_COMPUTE_CASE(12)
#endif
#if CT_NB > 13
    CT_COMPUTE_CASE(13)
#endif
#if CT_NB > 14
    CT_COMPUTE_CASE(14)
#endif
#if CT_NB > 15
    CT_COMPUTE_CASE(15)
#endif
    default: break;
    }
#undef CT_COMPUTE_CASE
}

// Persistent loop, two item buffers: while item k is computed from one, the
// copies of item k+1 into the other are in flight.  Work indices and item
// records rotate through three shared slots, so the slot thread 0 overwrites
// was last read two barriers earlier.  Thread 0 keeps the fetches off the
// block's critical path: the atomic that claims item k+2 is issued while
// item k starts (its result is first needed one item later), and item k+1's
// record is loaded before the barrier that precedes its staging.
#ifndef CT_MINB
#define CT_MINB 1
#endif
extern "C" __global__ void __launch_bounds__(CT_NT, CT_MINB) ct_corr2d_batch(const __grid_constant__ CtBatchParams p)
{
    extern __shared__ float4 ct_smem4[];
    __shared__ ct_u64 s_bar[2];
    __shared__ int s_w[3];
    __shared__ uint4 s_it[3];
    unsigned char* const raw = reinterpret_cast<unsigned char*>(ct_smem4);
    const ct_u32 mis = ct_sa(raw) & 127u;   // tensor copies land on 128-byte boundaries
    unsigned char* const buf0 = raw + (mis ? 128u - mis : 0u);
    unsigned char* const buf1 = buf0 + CT_BUF_BYTES;
    const int tid = threadIdx.x;
    ct_u32 fenced = 0xffffffffu;   // thread 0: problem whose tensor map it acquired last
    int claimed = 0;               // thread 0: the last index claimed (item k+1's at the top of iteration k)
    if (tid == 0) {
        ct_mbar_init(&s_bar[0], 1u);
        ct_mbar_init(&s_bar[1], 1u);
        ct_mbar_init_fence();
        const int w0 = (int)atomicAdd(p.counter, 1u);
        s_w[0] = w0;
        if (w0 < p.n_work) {
            const uint4 it = p.work[w0];
            s_it[0] = it;
            ct_stage_item(p, it, buf0, &s_bar[0], &fenced);
        }
        claimed = (int)atomicAdd(p.counter, 1u);
    }
    __syncthreads();
    ct_u32 phase = 0u;     // bit b: parity of buffer b's next completion
    ct_u32 pending = s_w[0] < p.n_work ? 1u : 0u;   // bit b: copies into buffer b started, not yet waited for
    int failed = 0;
    int slot = 0;   // s_w[slot] holds item k's index
    for (int k = 0;; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        const int nslot = slot == 2 ? 0 : slot + 1;
        uint4 it_next = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            const int wn = claimed;
            s_w[nslot] = wn;
            if (wn < p.n_work) it_next = p.work[wn];
            if (wn < p.n_work) claimed = (int)atomicAdd(p.counter, 1u);
        }
        // next index visible; every thread is done with the other buffer;
        // a timed-out wait in any thread stops the block
        if (__syncthreads_or(failed)) break;
        const int w = s_w[slot], wn = s_w[nslot];
        const int my = slot;
        slot = nslot;
        if (wn < p.n_work) {
            if (tid == 0) {
                s_it[nslot] = it_next;
                ct_stage_item(p, it_next, nxt ? buf1 : buf0, &s_bar[nxt], &fenced);
            }
            pending |= 1u << nxt;
        }
        if (w >= p.n_work) break;
        const bool ok = ct_mbar_wait(&s_bar[cur], (phase >> cur) & 1u);
        phase ^= 1u << cur;
        pending &= ~(1u << cur);
        if (!ok) {
            atomicOr(p.counter + 1, 1u);
            failed = 1;
            continue;
        }
        const uint4 it = s_it[my];
        ct_compute_item(p.probs[it.x], it.y, it.z, cur ? buf1 : buf0);
    }
    // copies can still be in flight only after a timed-out wait
    for (int b = 0; b < 2; ++b)
        if (pending & (1u << b)) (void)ct_mbar_wait(&s_bar[b], (phase >> b) & 1u);
}
