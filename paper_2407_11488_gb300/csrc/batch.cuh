// Persistent batched correlation: one launch works through a list of tiles
// that belong to many problems of uneven image and filter sizes.
//
// Compiled at run time by NVRTC to an sm_103a cubin.  Every problem belongs to
// a bucket (same filter size, similar image size); each bucket has its own
// compile-time tile routine (filter size, block shape, register tile), chosen
// by the library's tuner, and one launch holds all of them.  Each block
// repeatedly takes the next work item (problem, tile) from a global counter;
// the problem's filter taps and the tile's input halo are copied into one of
// two shared-memory buffers with cp.async while the block computes the
// previous item from the other buffer.
//
// The per-output arithmetic is that of the single-problem kernel: one FP32
// fused multiply-add per tap, taps added in (i, j) order, so results are
// bit-identical to ct_corr2d for the same inputs.
//
// Macros: CT_NT (threads per block), CT_DTYPE (0 FP32, 1 BF16 image),
// CT_NB (buckets), and for every bucket b < CT_NB: CT_B<b>_BX (block width;
// block height = CT_NT / BX), CT_B<b>_TX, CT_B<b>_TY (register tile),
// CT_B<b>_UN (1: input-row loop unrolled), CT_MINB (blocks per SM the
// register allocation must allow),
// CT_B<b>_FW, CT_B<b>_FH (filter); CT_BUF_FLOATS, the size of one item
// buffer (the largest bucket's, a multiple of 4 floats).
//
// Filters are stored FP32, each row padded with zeros to a multiple of 4
// taps, every filter starting on a 16-byte boundary.

#ifndef CT_DTYPE
#define CT_DTYPE 0
#endif

typedef long long ct_i64;
typedef unsigned int ct_u32;
#if CT_DTYPE == 0
typedef float ct_in_t;
#else
typedef unsigned short ct_in_t;
#endif

struct CtBatchProblem {
    const ct_in_t* in;
    float* out;
    ct_i64 in_pitch, out_pitch;
    int out_w, out_h, in_w, in_h;
    int bucket, tiles_x, filt_off, pad;
};

struct CtBatchParams {
    const CtBatchProblem* probs;
    const uint2* work;       // (problem index, tile index)
    const float* filters;    // all filters, FP32, rows padded to 4 taps, problem p at filt_off
    unsigned int* counter;   // next work item; zero before the launch
    int n_work;
};

__device__ __forceinline__ constexpr int ct_rup(int v, int m) { return (v + m - 1) / m * m; }

__device__ __forceinline__ void ct_cp16(float* dst, const void* src, bool valid)
{
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void ct_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ct_cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory buffer of one work item: filter taps (FH rows of FWP floats,
// zero padded), then the input tile plus halo (HH rows of SW floats).
// stage() and compute() are real calls, not inlined: each bucket's routine
// then gets its own register allocation and the kernel needs only the
// largest of them, instead of the union a single inlined body would hold.
template <int BX, int TX, int TY, int FW, int FH, int UN>
struct CtTile {
    static constexpr int BY = CT_NT / BX;
    static constexpr int TW = BX * TX, TH = BY * TY;
    static constexpr int HW = TW + FW - 1, HH = TH + FH - 1;
    static constexpr int SW = ct_rup(HW, 4);
    static constexpr int FWP = ct_rup(FW, 4);
    static constexpr int VW = (TX % 4 == 0) ? 4 : ((TX % 2 == 0) ? 2 : 1);
    static constexpr int WW = TX + FW - 1;
    static constexpr int WWV = ct_rup(WW, VW);

    // Starts the copies of one item into buf (asynchronous for FP32 images).
    static __device__ __noinline__ void stage(const CtBatchProblem& pr, const float* __restrict__ filters,
                                                 int tile, float* buf)
    {
        const int tid = threadIdx.x;
        float* taps = buf;
        float* halo = buf + FH * FWP;
        const int gx0 = (tile % pr.tiles_x) * TW, gy0 = (tile / pr.tiles_x) * TH;
        for (int k = tid; k < FH * FWP / 4; k += CT_NT) ct_cp16(taps + 4 * k, filters + pr.filt_off + 4 * k, true);
        constexpr int CH = SW / 4;
        constexpr int NCH = HH * CH;
#pragma unroll 4
        for (int idx = tid; idx < NCH; idx += CT_NT) {
            const int r = idx / CH;
            const int c = (idx - r * CH) * 4;
            const int yy = gy0 + r, xx = gx0 + c;
            const bool ok = yy < pr.in_h && xx < pr.in_w;
#if CT_DTYPE == 0
            ct_cp16(halo + r * SW + c, ok ? (const void*)(pr.in + (ct_i64)yy * pr.in_pitch + xx) : (const void*)pr.in,
                    ok);
#else
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (ok) {
                const uint2 u = __ldg(reinterpret_cast<const uint2*>(pr.in + (ct_i64)yy * pr.in_pitch + xx));
                v = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
            }
            *reinterpret_cast<float4*>(halo + r * SW + c) = v;
#endif
        }
    }

    static __device__ __forceinline__ void row_step(const float* halo, const float* taps, int lx, int ly, int r,
                                                    float (&acc)[TY][TX])
    {
        const float* s = halo + (ly + r) * SW + lx;
        float w[WWV];
#pragma unroll
        for (int k = 0; k < WWV; k += VW) {
            if (VW == 4) {
                const float4 v = *reinterpret_cast<const float4*>(s + k);
                w[k] = v.x; w[k + 1] = v.y; w[k + 2] = v.z; w[k + 3] = v.w;
            } else if (VW == 2) {
                const float2 v = *reinterpret_cast<const float2*>(s + k);
                w[k] = v.x; w[k + 1] = v.y;
            } else {
                w[k] = s[k];
            }
        }
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

    // Computes and stores one item whose taps and halo are in buf.
    static __device__ __noinline__ void compute(const CtBatchProblem& pr, int tile, const float* buf)
    {
        const int tid = threadIdx.x;
        const float* taps = buf;
        const float* halo = buf + FH * FWP;
        const int gx0 = (tile % pr.tiles_x) * TW, gy0 = (tile / pr.tiles_x) * TH;
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

__device__ __forceinline__ void ct_stage_item(const CtBatchProblem& pr, const float* filters, int tile, float* buf)
{
    switch (pr.bucket) {
#if CT_NB > 0
    case 0: CT_TILE(0)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 1
    case 1: CT_TILE(1)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 2
    case 2: CT_TILE(2)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 3
    case 3: CT_TILE(3)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 4
    case 4: CT_TILE(4)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 5
    case 5: CT_TILE(5)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 6
    case 6: CT_TILE(6)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 7
    case 7: CT_TILE(7)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 8
    case 8: CT_TILE(8)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 9
    case 9: CT_TILE(9)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 10
    case 10: CT_TILE(10)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 11
    case 11: CT_TILE(11)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 12
    case 12: CT_TILE(12)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 13
    case 13: CT_TILE(13)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 14
    case 14: CT_TILE(14)::stage(pr, filters, tile, buf); break;
#endif
#if CT_NB > 15
    case 15: CT_TILE(15)::stage(pr, filters, tile, buf); break;
#endif
    default: break;
    }
}

__device__ __forceinline__ void ct_compute_item(const CtBatchProblem& pr, int tile, const float* buf)
{
    switch (pr.bucket) {
#if CT_NB > 0
    case 0: CT_TILE(0)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 1
    case 1: CT_TILE(1)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 2
    case 2: CT_TILE(2)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 3
    case 3: CT_TILE(3)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 4
    case 4: CT_TILE(4)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 5
    case 5: CT_TILE(5)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 6
    case 6: CT_TILE(6)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 7
    case 7: CT_TILE(7)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 8
    case 8: CT_TILE(8)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 9
    case 9: CT_TILE(9)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 10
    case 10: CT_TILE(10)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 11
    case 11: CT_TILE(11)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 12
    case 12: CT_TILE(12)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 13
    case 13: CT_TILE(13)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 14
    case 14: CT_TILE(14)::compute(pr, tile, buf); break;
#endif
#if CT_NB > 15
    case 15: CT_TILE(15)::compute(pr, tile, buf); break;
#endif
    default: break;
    }
}

// Persistent loop, two shared buffers: while item k is computed from one, the
// copies of item k+1 into the other are in flight.
#ifndef CT_MINB
#define CT_MINB 1
#endif
extern "C" __global__ void __launch_bounds__(CT_NT, CT_MINB) ct_corr2d_batch(const __grid_constant__ CtBatchParams p)
{
    extern __shared__ float4 ct_smem4[];
    float* const sm0 = reinterpret_cast<float*>(ct_smem4);
    float* const sm1 = sm0 + CT_BUF_FLOATS;
    __shared__ int s_w[2];
    const int tid = threadIdx.x;
    if (tid == 0) s_w[0] = (int)atomicAdd(p.counter, 1u);
    __syncthreads();
    {
        const int w0 = s_w[0];
        if (w0 < p.n_work) {
            const uint2 it = p.work[w0];
            ct_stage_item(p.probs[it.x], p.filters, (int)it.y, sm0);
        }
        ct_cp_commit();
    }
    for (int k = 0;; ++k) {
        const int cur = k & 1;
        float* const bcur = cur ? sm1 : sm0;
        float* const bnxt = cur ? sm0 : sm1;
        if (tid == 0) s_w[cur ^ 1] = (int)atomicAdd(p.counter, 1u);
        __syncthreads();   // next index visible; every thread is done with bnxt
        const int w = s_w[cur];
        const int wn = s_w[cur ^ 1];
        if (wn < p.n_work) {
            const uint2 it = p.work[wn];
            ct_stage_item(p.probs[it.x], p.filters, (int)it.y, bnxt);
        }
        ct_cp_commit();
        ct_cp_wait<1>();   // this thread's copies of item w have landed
        __syncthreads();   // ... and every other thread's
        if (w >= p.n_work) break;
        const uint2 it = p.work[w];
        ct_compute_item(p.probs[it.x], (int)it.y, bcur);
    }
    ct_cp_wait<0>();
}
