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
// CT_B<b>_UN (1: input-row loop unrolled), CT_B<b>_FW, CT_B<b>_FH (filter);
// CT_MINB (blocks per SM the register allocation must allow); CT_BUF_BYTES,
// the size of one item buffer (the largest bucket's, a multiple of 128).
//
// Filters are stored FP32, each row padded with zeros to a multiple of 4
// taps, every filter starting on a 16-byte boundary.  Waits on an mbarrier
// give up after about two seconds: the block then sets bit 0 of counter[1],
// waits (again bounded) for the copies it started, and exits.

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
    const uint2* work;            // (problem index, (tile row << 16) | tile column)
    const float* filters;         // all filters, FP32, rows padded to 4 taps, problem p at filt_off
    const unsigned char* tmaps;   // problem p's tensor map (128 bytes) at tmaps + 128 p
    unsigned int* counter;        // [0]: next work item, zero before the launch; [1]: error bits
    int n_work;
};

__device__ __forceinline__ constexpr int ct_rup(int v, int m) { return (v + m - 1) / m * m; }

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
template <int BX, int TX, int TY, int FW, int FH, int UN>
struct CtTile {
    static constexpr int BY = CT_NT / BX;
    static constexpr int TW = BX * TX, TH = BY * TY;
    static constexpr int HW = TW + FW - 1, HH = TH + FH - 1;
    static constexpr int SW = ct_rup(HW, CT_BOXQ);
    static constexpr int FWP = ct_rup(FW, 4);
    static constexpr int HALO_BYTES = HH * SW * CT_ESZ;
    static constexpr int TAPS_OFF = ct_rup(HALO_BYTES, 16);
    static constexpr int TAP_BYTES = FH * FWP * 4;
    static constexpr int VW = (TX % 4 == 0) ? 4 : ((TX % 2 == 0) ? 2 : 1);
    static constexpr int WW = TX + FW - 1;
    static constexpr int WWV = ct_rup(WW, VW);
    static_assert(SW <= 256 && HH <= 256, "the halo box exceeds 256 elements per side");
    static_assert(ct_rup(TAPS_OFF + TAP_BYTES, 128) <= CT_BUF_BYTES, "item buffer too small");
    static_assert(TW % 16 == 0, "tile columns must start on 16-element boundaries");

    // Thread 0: starts both copies of one item into buf, completing on bar.
    static __device__ __forceinline__ void stage(const CtBatchProblem& pr, const unsigned char* tmap,
                                                 const float* filters, ct_u32 tile, unsigned char* buf, ct_u64* bar)
    {
        const int gx0 = (int)(tile & 0xffffu) * TW, gy0 = (int)(tile >> 16) * TH;
        ct_tmap_acquire(tmap);
        ct_mbar_expect_tx(bar, (ct_u32)(HALO_BYTES + TAP_BYTES + CT_TEST_EXTRA_TX));
        ct_tma_load_2d(buf, tmap, gx0, gy0, bar);
        ct_bulk_load(buf + TAPS_OFF, filters + pr.filt_off, (ct_u32)TAP_BYTES, bar);
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
        if constexpr (UN != 0) {
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

#define CT_TILE(b) CtTile<CT_B##b##_BX, CT_B##b##_TX, CT_B##b##_TY, CT_B##b##_FW, CT_B##b##_FH, CT_B##b##_UN>

// Thread 0: starts the copies of work item w into buf.
__device__ __forceinline__ void ct_stage_item(const CtBatchParams& p, int w, unsigned char* buf, ct_u64* bar)
{
    const uint2 it = p.work[w];
    const CtBatchProblem& pr = p.probs[it.x];
    const unsigned char* tmap = p.tmaps + 128ull * it.x;
#define CT_STAGE_CASE(b) \
    case b: CT_TILE(b)::stage(pr, tmap, p.filters, it.y, buf, bar); break;
    switch (pr.bucket) {
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

__device__ __forceinline__ void ct_compute_item(const CtBatchProblem& pr, ct_u32 tile, const unsigned char* buf)
{
#define CT_COMPUTE_CASE(b) \
    case b: CT_TILE(b)::compute(pr, tile, buf); break;
    switch (pr.bucket) {
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
// copies of item k+1 into the other are in flight.  Work indices rotate
// through three shared slots, so the slot thread 0 overwrites was last read
// two barriers earlier.
#ifndef CT_MINB
#define CT_MINB 1
#endif
extern "C" __global__ void __launch_bounds__(CT_NT, CT_MINB) ct_corr2d_batch(const __grid_constant__ CtBatchParams p)
{
    extern __shared__ float4 ct_smem4[];
    __shared__ ct_u64 s_bar[2];
    __shared__ int s_w[3];
    unsigned char* const raw = reinterpret_cast<unsigned char*>(ct_smem4);
    const ct_u32 mis = ct_sa(raw) & 127u;   // tensor copies land on 128-byte boundaries
    unsigned char* const buf0 = raw + (mis ? 128u - mis : 0u);
    unsigned char* const buf1 = buf0 + CT_BUF_BYTES;
    const int tid = threadIdx.x;
    if (tid == 0) {
        ct_mbar_init(&s_bar[0], 1u);
        ct_mbar_init(&s_bar[1], 1u);
        ct_mbar_init_fence();
        s_w[0] = (int)atomicAdd(p.counter, 1u);
    }
    __syncthreads();
    ct_u32 phase = 0u;     // bit b: parity of buffer b's next completion
    ct_u32 pending = 0u;   // bit b: copies into buffer b started and not yet waited for
    int failed = 0;
    if (s_w[0] < p.n_work) {
        if (tid == 0) ct_stage_item(p, s_w[0], buf0, &s_bar[0]);
        pending = 1u;
    }
    int slot = 0;   // s_w[slot] holds item k's index
    for (int k = 0;; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        const int nslot = slot == 2 ? 0 : slot + 1;
        if (tid == 0) s_w[nslot] = (int)atomicAdd(p.counter, 1u);
        // next index visible; every thread is done with the other buffer;
        // a timed-out wait in any thread stops the block
        if (__syncthreads_or(failed)) break;
        const int w = s_w[slot], wn = s_w[nslot];
        slot = nslot;
        if (wn < p.n_work) {
            if (tid == 0) ct_stage_item(p, wn, nxt ? buf1 : buf0, &s_bar[nxt]);
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
        const uint2 it = p.work[w];
        ct_compute_item(p.probs[it.x], it.y, cur ? buf1 : buf0);
    }
    // copies can still be in flight only after a timed-out wait
    for (int b = 0; b < 2; ++b)
        if (pending & (1u << b)) (void)ct_mbar_wait(&s_bar[b], (phase >> b) & 1u);
}
