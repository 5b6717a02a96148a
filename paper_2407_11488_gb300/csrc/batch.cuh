// Persistent batched correlation: one launch works through a list of tiles
// that belong to many problems of uneven image and filter sizes.
//
// Compiled at run time by NVRTC to an sm_103a cubin.  Every problem belongs to
// a bucket (same filter size, similar image size); each bucket has its own
// compile-time tile routine (filter size, block shape, register tile), chosen
// by the library's tuner, and one launch holds all of them.  Each block
// repeatedly takes the next work item (problem, tile) from a global counter,
// stages the problem's filter taps and the tile's input halo in shared
// memory, computes the tile and stores it.
//
// The per-output arithmetic is that of the single-problem kernel: one FP32
// fused multiply-add per tap, taps added in (i, j) order, so results are
// bit-identical to ct_corr2d for the same inputs.
//
// Macros: CT_NT (threads per block), CT_DTYPE (0 FP32, 1 BF16 image),
// CT_NB (buckets), and for every bucket b < CT_NB: CT_B<b>_BX (block width;
// block height = CT_NT / BX), CT_B<b>_TX, CT_B<b>_TY (register tile),
// CT_B<b>_FW, CT_B<b>_FH (filter).

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
    const float* filters;    // all filters, FP32, row-major, problem p at filt_off
    unsigned int* counter;   // next work item; zero before the launch
    int n_work;
};

__device__ __forceinline__ constexpr int ct_rup(int v, int m) { return (v + m - 1) / m * m; }

template <int BX, int TX, int TY, int FW, int FH>
__device__ __forceinline__ void ct_batch_tile(const CtBatchProblem& pr, const float* __restrict__ filters, int tile,
                                              float* sm)
{
    constexpr int BY = CT_NT / BX;
    constexpr int TW = BX * TX, TH = BY * TY;
    constexpr int HW = TW + FW - 1, HH = TH + FH - 1;
    constexpr int SW = ct_rup(HW, 4);
    constexpr int FWP = ct_rup(FW, 4);
    constexpr int VW = (TX % 4 == 0) ? 4 : ((TX % 2 == 0) ? 2 : 1);
    constexpr int WW = TX + FW - 1;
    constexpr int WWV = ct_rup(WW, VW);
    float* taps = sm;
    float* halo = sm + FH * FWP;

    const int tid = threadIdx.x;
    const int bxi = tile % pr.tiles_x, byi = tile / pr.tiles_x;
    const int gx0 = bxi * TW, gy0 = byi * TH;

    // filter taps, rows padded to a multiple of 4 with zeros
    for (int k = tid; k < FH * FWP; k += CT_NT) {
        const int i = k / FWP, j = k - i * FWP;
        taps[k] = j < FW ? __ldg(filters + pr.filt_off + i * FW + j) : 0.0f;
    }
    // input tile plus halo in 4-element chunks (16 bytes FP32, 8 bytes BF16)
    {
        constexpr int CH = SW / 4;
        constexpr int NCH = HH * CH;
#pragma unroll 4
        for (int idx = tid; idx < NCH; idx += CT_NT) {
            const int r = idx / CH;
            const int c = (idx - r * CH) * 4;
            const int yy = gy0 + r, xx = gx0 + c;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (yy < pr.in_h && xx < pr.in_w) {
                const ct_in_t* src = pr.in + (ct_i64)yy * pr.in_pitch + xx;
#if CT_DTYPE == 0
                v = __ldg(reinterpret_cast<const float4*>(src));
#else
                const uint2 u = __ldg(reinterpret_cast<const uint2*>(src));
                v = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
#endif
            }
            *reinterpret_cast<float4*>(halo + r * SW + c) = v;
        }
    }
    __syncthreads();

    const int lx = (tid % BX) * TX, ly = (tid / BX) * TY;
    float acc[TY][TX];
#pragma unroll
    for (int ty = 0; ty < TY; ++ty)
#pragma unroll
        for (int tx = 0; tx < TX; ++tx) acc[ty][tx] = 0.0f;

#pragma unroll 1
    for (int i = 0; i < FH; ++i) {
        float f[FWP];
#pragma unroll
        for (int q = 0; q < FWP; q += 4) {
            const float4 t = *reinterpret_cast<const float4*>(taps + i * FWP + q);
            f[q] = t.x; f[q + 1] = t.y; f[q + 2] = t.z; f[q + 3] = t.w;
        }
#pragma unroll
        for (int ty = 0; ty < TY; ++ty) {
            const float* s = halo + (ly + ty + i) * SW + lx;
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
            for (int j = 0; j < FW; ++j)
#pragma unroll
                for (int tx = 0; tx < TX; ++tx) acc[ty][tx] = fmaf(w[tx + j], f[j], acc[ty][tx]);
        }
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
    __syncthreads();   // the next item re-stages shared memory
}

#define CT_BUCKET_CASE(b)                                                                                  \
    case b:                                                                                                \
        ct_batch_tile<CT_B##b##_BX, CT_B##b##_TX, CT_B##b##_TY, CT_B##b##_FW, CT_B##b##_FH>(pr, p.filters, \
                                                                                           it.y, sm);     \
        break;

extern "C" __global__ void __launch_bounds__(CT_NT) ct_corr2d_batch(const __grid_constant__ CtBatchParams p)
{
    extern __shared__ float4 ct_smem4[];
    float* sm = reinterpret_cast<float*>(ct_smem4);
    __shared__ int s_w;
    for (;;) {
        if (threadIdx.x == 0) s_w = (int)atomicAdd(p.counter, 1u);
        __syncthreads();
        const int w = s_w;
        if (w >= p.n_work) break;
        const uint2 it = p.work[w];
        const CtBatchProblem pr = p.probs[it.x];
        switch (pr.bucket) {
#if CT_NB > 0
            CT_BUCKET_CASE(0)
#endif
#if CT_NB > 1
            CT_BUCKET_CASE(1)
#endif
#if CT_NB > 2
            CT_BUCKET_CASE(2)
#endif
#if CT_NB > 3
            CT_BUCKET_CASE(3)
#endif
#if CT_NB > 4
            CT_BUCKET_CASE(4)
#endif
#if CT_NB > 5
            CT_BUCKET_CASE(5)
#endif
#if CT_NB > 6
            CT_BUCKET_CASE(6)
#endif
#if CT_NB > 7
            CT_BUCKET_CASE(7)
#endif
#if CT_NB > 8
            CT_BUCKET_CASE(8)
#endif
#if CT_NB > 9
            CT_BUCKET_CASE(9)
#endif
#if CT_NB > 10
            CT_BUCKET_CASE(10)
#endif
#if CT_NB > 11
            CT_BUCKET_CASE(11)
#endif
#if CT_NB > 12
            CT_BUCKET_CASE(12)
#endif
#if CT_NB > 13
            CT_BUCKET_CASE(13)
#endif
#if CT_NB > 14
            CT_BUCKET_CASE(14)
#endif
#if CT_NB > 15
            CT_BUCKET_CASE(15)
#endif
            default: __syncthreads(); break;
        }
    }
}
