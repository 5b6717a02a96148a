// Direct single-channel 2D correlation, one tunable variant per compilation.
//
// This source is compiled at run time by NVRTC straight to an sm_103a cubin
// (one cubin per point of the search space and filter size), the way an
// empirical auto-tuner compiles and benchmarks each configuration of a
// tunable kernel (Sec. 3 "Design and Implementation"; the tunable parameters
// of the 2D convolution kernel are Table 1's block_size_x/y, tile_size_x/y,
// use_shmem, plus the loop-unrolling switch of Sec. 3).
//
// Computes the valid cross-correlation
//     out[y][x] = sum_{i<FH} sum_{j<FW} in[y+i][x+j] * f[i][j]
// in FP32 with one fused multiply-add per tap.  Every variant adds the taps of
// one output in the same order (i ascending, then j ascending), so all points
// of the space give bit-identical results.
//
// Compile-time parameters (macros):
//   CT_BX, CT_BY   thread-block shape (threads in x and y)
//   CT_TX, CT_TY   outputs per thread in x and y (register tile)
//   CT_SMEM        0: each thread reads its input window from global memory
//                     (through L1);
//                  1: the block stages its input tile plus halo in shared
//                     memory, then reads windows from there
//   CT_TMA         (chosen by the host with CT_SMEM = 1 when the halo box is
//                  at most 256 x 256 elements: for FP32 images, and for BF16
//                  images in the paired form) 1: one thread stages the halo
//                  with a 2D tensor copy (the tensor map in the parameter
//                  block; elements outside the image arrive as zeros) that
//                  completes on an mbarrier; a BF16 halo stays BF16 in shared
//                  memory and is widened as a row enters registers.  0: every
//                  thread copies 16-byte chunks (BF16 widened to FP32 on the way)
//   CT_UNROLL      1: fully unrolled; input rows slide through a register
//                     window and each row feeds every output row that uses it;
//                  0: the loop over filter rows stays rolled; 2, 4: that loop
//                     is unrolled by this factor (partial unrolling)
//   CT_FW, CT_FH   filter width and height
//   CT_DTYPE       0: FP32 image; 1: BF16 image (widened to FP32 on load)
//   CT_TAPS_IMM    1 (with CT_UNROLL = 1): the taps are compiled in, from
//                  CT_TAP_VALUES (FH*FW float literals, row-major), so every
//                  multiply-add takes its tap as an immediate operand; 0: the
//                  taps come from the parameter block
//   CT_SHFL        1 (with CT_SMEM = 1, CT_BX a multiple of 32, CT_TX a
//                  multiple of 4): a thread reads only its own TX values of an
//                  input row from shared memory and takes the other WW - TX
//                  values of its window from the lanes to its right with warp
//                  shuffles (a warp is 32 consecutive threads of one thread
//                  row); a lane whose window runs past the warp's last lane
//                  then reads its whole window itself.  The same values reach
//                  the same registers, so the bits are unchanged
//   CT_FMA2        1 (with CT_UNROLL = 1, CT_TY >= 2, CT_TAPS_IMM = 0): output
//                  rows 2k and 2k+1 of a thread pair up; an input row feeds
//                  both through one paired FP32 multiply-add (fma.rn.f32x2)
//                  per column and tap, with the tap pair (f[i][j], f[i-1][j])
//                  from the parameter block.  Each half is an ordinary fma.rn,
//                  and every output still adds its taps in (i, j) order, so
//                  the bits are those of the scalar form
//
// Layout contract (checked by the host before launch): row pitches are in
// elements and make every row start on a 16-byte boundary; the image buffer
// holds in_h full rows of in_pitch elements; the filter taps travel by value
// in the kernel's parameter block (constant bank), so FFMAs take them as
// uniform operands with no load instruction.  A wait for the tensor copy
// gives up after about two seconds: the block then sets bit 0 of the error
// word, waits (again bounded) for the copy, and stores nothing more.
//
// Grid (a launch-time choice, the same cubin): either one block per output
// tile (a 2-D grid of tiles_x x tiles_y blocks), or persistent (p.persist = 1:
// a 1-D grid of as many blocks as the GPU holds at once; block b computes
// tiles b, b + G, b + 2G, ... in row-major tile order, G = gridDim.x), which
// spreads the last partial wave of tiles evenly over the SMs.

#ifndef CT_DTYPE
#define CT_DTYPE 0
#endif
#ifndef CT_TMA
#define CT_TMA 0
#endif
#ifndef CT_FMA2
#define CT_FMA2 0
#endif
#if CT_TMA && CT_DTYPE != 0 && !CT_FMA2
#error "BF16 images are staged by a tensor copy in the paired form only"
#endif
// Test hook: bytes expected on top of those the tensor copy delivers; a
// nonzero value makes the wait run out.  0 in every normal build.
#ifndef CT_TEST_EXTRA_TX
#define CT_TEST_EXTRA_TX 0
#endif

#ifndef CT_TAPS_IMM
#define CT_TAPS_IMM 0
#endif
#if CT_TAPS_IMM && CT_UNROLL != 1
#error "compiled-in taps need the unrolled body"
#endif
#if CT_FMA2 && (CT_UNROLL != 1 || CT_TY < 2 || CT_TAPS_IMM)
#error "paired multiply-adds need the unrolled body, two output rows per thread and parameter-block taps"
#endif
#ifndef CT_SHFL
#define CT_SHFL 0
#endif
#if CT_SHFL && (!CT_SMEM || CT_BX % 32 != 0 || CT_TX % 4 != 0 || (CT_TMA && CT_DTYPE != 0))
#error "shuffled windows need shared-memory staging, whole warps per thread row and 4-wide register tiles"
#endif

#ifdef CT_INJECT_COMPILE_ERROR
#error "compile failure requested through CT_INJECT_COMPILE_ERROR"
#endif

typedef long long ct_i64;
typedef unsigned int ct_u32;
typedef unsigned long long ct_u64;

#if CT_DTYPE == 0
typedef float ct_in_t;
#else
typedef unsigned short ct_in_t;
#endif

struct __align__(64) CtTensorMap {
    unsigned long long q[16];
};

struct CtParams {
    CtTensorMap tmap;   // the image's tensor map (CT_TMA variants; zero otherwise)
    const ct_in_t* in;
    float* out;
    ct_i64 in_pitch;
    ct_i64 out_pitch;
    int out_w, out_h;
    int in_w, in_h;
    unsigned* err;      // error word
    int tiles_x;        // tile columns
    int n_tiles;        // tiles in all
    int persist;        // 1: persistent 1-D grid (see above)
    int step_x, step_y; // persistent: gridDim.x as (tile columns, tile rows) of the row-major order
    int pad_;
    float f[CT_FH * CT_FW];
#if CT_FMA2
    ct_u64 fp[CT_FH * CT_FW];   // entry i*FW+j, i >= 1: f[i][j] in the low half, f[i-1][j] in the high half
#endif
};

#define CT_NT (CT_BX * CT_BY)
#define CT_WW (CT_TX + CT_FW - 1)
#define CT_TILE_W (CT_BX * CT_TX)
#define CT_TILE_H (CT_BY * CT_TY)
#define CT_HALO_W (CT_TILE_W + CT_FW - 1)
#define CT_HALO_H (CT_TILE_H + CT_FH - 1)
#if CT_TMA && CT_DTYPE != 0
typedef ct_in_t ct_st_t;                     // the staged element: BF16 halos stay BF16
#define CT_SW (((CT_HALO_W + 7) / 8) * 8)    // staged row length in elements (the tensor-copy box width)
#else
typedef float ct_st_t;
#define CT_SW (((CT_HALO_W + 3) / 4) * 4)    // staged row length in elements (the tensor-copy box width)
#endif

#if CT_TX % 4 == 0
#define CT_VW 4
#elif CT_TX % 2 == 0
#define CT_VW 2
#else
#define CT_VW 1
#endif
#define CT_WWV (((CT_WW + CT_VW - 1) / CT_VW) * CT_VW)

__device__ __forceinline__ float ct_bf16(unsigned short h)
{
    return __uint_as_float(((ct_u32)h) << 16);
}

// Loads VW consecutive input elements starting at p (aligned to VW elements).
template <int VW>
__device__ __forceinline__ void ct_ldg(float* w, const ct_in_t* __restrict__ p)
{
#if CT_DTYPE == 0
    if (VW == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if (VW == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
        w[0] = __ldg(p);
    }
#else
    if (VW == 4) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        w[0] = __uint_as_float(v.x << 16); w[1] = __uint_as_float(v.x & 0xffff0000u);
        w[2] = __uint_as_float(v.y << 16); w[3] = __uint_as_float(v.y & 0xffff0000u);
    } else if (VW == 2) {
        const ct_u32 v = __ldg(reinterpret_cast<const unsigned int*>(p));
        w[0] = __uint_as_float(v << 16); w[1] = __uint_as_float(v & 0xffff0000u);
    } else {
        w[0] = ct_bf16(__ldg(p));
    }
#endif
}

// One input row of the thread's window: columns gx .. gx+CT_WWV-1 of row gy.
// Chunks that start at or beyond in_w (or rows beyond in_h) read as zero; a
// chunk that starts inside the row may run into the row's padding, which
// only feeds outputs at x >= out_w (never stored).
__device__ __forceinline__ void ct_row_global(float (&w)[CT_WWV], const CtParams& p, int gy, int gx)
{
    if (gy < p.in_h) {
        const ct_in_t* __restrict__ row = p.in + (ct_i64)gy * p.in_pitch + gx;
#pragma unroll
        for (int k = 0; k < CT_WWV; k += CT_VW) {
            if (gx + k < p.in_w) {
                ct_ldg<CT_VW>(w + k, row + k);
            } else {
#pragma unroll
                for (int e = 0; e < CT_VW; ++e) w[k + e] = 0.0f;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < CT_WWV; ++k) w[k] = 0.0f;
    }
}

#if CT_TMA
__device__ __forceinline__ unsigned ct_sa(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// One test of the barrier phase; a thread whose phase has not completed is
// suspended until it does or up to about 0.1 ms (the suspend-time hint), so
// a waiting warp issues few instructions.
__device__ __forceinline__ bool ct_bar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(ct_sa(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return done != 0;
}
// Waits for phase `parity` of bar; false after about two seconds.
__device__ __forceinline__ bool ct_bar_wait(unsigned long long* bar, unsigned parity)
{
    if (ct_bar_try_wait(bar, parity)) return true;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t0));
    for (;;) {
        if (ct_bar_try_wait(bar, parity)) return true;
        asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
        if (t - t0 > 2000000000ull) return false;
    }
}

#endif

#if CT_FMA2
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
// d = a * b + c in each half, each an fma.rn.f32
__device__ __forceinline__ ct_u64 ct_fma2(ct_u64 a, ct_u64 b, ct_u64 c)
{
    ct_u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
#endif

// A staged BF16 row: VW consecutive elements per load, widened exactly.
__device__ __forceinline__ void ct_row_shared(float (&w)[CT_WWV], const unsigned short* __restrict__ s)
{
#pragma unroll
    for (int k = 0; k < CT_WWV; k += CT_VW) {
        if (CT_VW == 4) {
            const uint2 v = *reinterpret_cast<const uint2*>(s + k);
            w[k] = __uint_as_float(v.x << 16); w[k + 1] = __uint_as_float(v.x & 0xffff0000u);
            w[k + 2] = __uint_as_float(v.y << 16); w[k + 3] = __uint_as_float(v.y & 0xffff0000u);
        } else if (CT_VW == 2) {
            const ct_u32 v = *reinterpret_cast<const ct_u32*>(s + k);
            w[k] = __uint_as_float(v << 16); w[k + 1] = __uint_as_float(v & 0xffff0000u);
        } else {
            w[k] = __uint_as_float(((ct_u32)s[k]) << 16);
        }
    }
}

__device__ __forceinline__ void ct_row_shared(float (&w)[CT_WWV], const float* __restrict__ s)
{
#pragma unroll
    for (int k = 0; k < CT_WWV; k += CT_VW) {
        if (CT_VW == 4) {
            const float4 v = *reinterpret_cast<const float4*>(s + k);
            w[k] = v.x; w[k + 1] = v.y; w[k + 2] = v.z; w[k + 3] = v.w;
        } else if (CT_VW == 2) {
            const float2 v = *reinterpret_cast<const float2*>(s + k);
            w[k] = v.x; w[k + 1] = v.y;
        } else {
            w[k] = s[k];
        }
    }
}

#if CT_SHFL
// The window of a lane from its own TX values and its right-hand neighbours'
// (lane + d holds columns d*TX .. d*TX+TX-1 past this lane's first column).
__device__ __forceinline__ void ct_row_shfl(float (&w)[CT_WWV], const float* __restrict__ s, unsigned lane)
{
#pragma unroll
    for (int k = 0; k < CT_TX; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(s + k);
        w[k] = v.x; w[k + 1] = v.y; w[k + 2] = v.z; w[k + 3] = v.w;
    }
#pragma unroll
    for (int m = 0; m < CT_WW - CT_TX; ++m)
        w[CT_TX + m] = __shfl_down_sync(0xffffffffu, w[m % CT_TX], 1 + m / CT_TX);
    if (lane + (CT_WW - 1) / CT_TX > 31u) ct_row_shared(w, s);   // past the warp: read it all
}
#endif

extern "C" __global__ void __launch_bounds__(CT_NT)
ct_corr2d(const __grid_constant__ CtParams p)
{
    const int lx = threadIdx.x * CT_TX;
    const int ly = threadIdx.y * CT_TY;
    // this block's first tile
    int txi = blockIdx.x, tyi = blockIdx.y;
    if (p.persist) {
        tyi = blockIdx.x / p.tiles_x;
        txi = blockIdx.x - tyi * p.tiles_x;
    }
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
#if CT_TAPS_IMM
    constexpr float ct_taps[CT_FH * CT_FW] = {CT_TAP_VALUES};
#define CT_TAP(k) ct_taps[k]
#else
#define CT_TAP(k) p.f[k]
#endif

#if CT_SHFL
    const unsigned lane = threadIdx.x & 31u;
#define CT_ROW_SMEM(w, s) ct_row_shfl(w, s, lane)
#else
#define CT_ROW_SMEM(w, s) ct_row_shared(w, s)
#endif
#if CT_SMEM && CT_TMA
    extern __shared__ float4 ct_smem4[];
    __shared__ unsigned long long ct_bar;
    unsigned char* const raw = reinterpret_cast<unsigned char*>(ct_smem4);
    const unsigned mis = ct_sa(raw) & 127u;   // the tensor copy lands on a 128-byte boundary
    ct_st_t* const sm = reinterpret_cast<ct_st_t*>(raw + (mis ? 128u - mis : 0u));
    if (lead) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ct_sa(&ct_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();   // the barrier is initialised before anyone waits on it
    unsigned phase = 0u;
#define CT_LOAD_ROW(w, r) CT_ROW_SMEM(w, sm + (ly + (r)) * CT_SW + lx)
#elif CT_SMEM
    extern __shared__ float4 ct_smem4[];
    float* sm = reinterpret_cast<float*>(ct_smem4);
#define CT_LOAD_ROW(w, r) CT_ROW_SMEM(w, sm + (ly + (r)) * CT_SW + lx)
#else
#define CT_LOAD_ROW(w, r) ct_row_global(w, p, gy + (r), gx)
#endif

    for (int t = p.persist ? (int)blockIdx.x : 0;;) {
        const int gx0 = txi * CT_TILE_W;
        const int gy0 = tyi * CT_TILE_H;
        const int gx = gx0 + lx;
        const int gy = gy0 + ly;
        bool ok = true;

#if CT_SMEM && CT_TMA
        if (lead) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(ct_sa(&ct_bar)),
                         "r"((unsigned)(CT_HALO_H * CT_SW * sizeof(ct_st_t) + CT_TEST_EXTRA_TX))
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                "%3}], [%4];\n" ::"r"(ct_sa(sm)),
                "l"(&p.tmap), "r"(gx0), "r"(gy0), "r"(ct_sa(&ct_bar))
                : "memory");
        }
        ok = ct_bar_wait(&ct_bar, phase);
        if (!ok) {
            atomicOr(p.err, 1u);
            if (lead) (void)ct_bar_wait(&ct_bar, phase);   // the copy may still land: wait (bounded) before leaving
        }
        phase ^= 1u;
#elif CT_SMEM
        {
            // Stage rows gy0 .. gy0+HALO_H-1, columns gx0 .. gx0+SW-1 in 4-element
            // chunks (16 bytes for FP32, 8 for BF16).  gx0 is a multiple of 16.
            constexpr int CH = CT_SW / 4;
            constexpr int NCH = CT_HALO_H * CH;
            const int tid = threadIdx.y * CT_BX + threadIdx.x;
#pragma unroll 4
            for (int idx = tid; idx < NCH; idx += CT_NT) {
                const int r = idx / CH;
                const int c = (idx - r * CH) * 4;
                const int yy = gy0 + r, xx = gx0 + c;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (yy < p.in_h && xx < p.in_w) {
                    const ct_in_t* src = p.in + (ct_i64)yy * p.in_pitch + xx;
#if CT_DTYPE == 0
                    v = __ldg(reinterpret_cast<const float4*>(src));
#else
                    const uint2 u = __ldg(reinterpret_cast<const uint2*>(src));
                    v = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                    __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
#endif
                }
                *reinterpret_cast<float4*>(sm + r * CT_SW + c) = v;
            }
        }
        __syncthreads();
#endif

        if (ok) {
            float acc[CT_TY][CT_TX];
#pragma unroll
            for (int ty = 0; ty < CT_TY; ++ty)
#pragma unroll
                for (int tx = 0; tx < CT_TX; ++tx) acc[ty][tx] = 0.0f;

#if CT_UNROLL == 1 && CT_FMA2
            // Output rows 2k and 2k+1 pair up: input row r feeds them with
            // filter rows i = r - 2k and i - 1.  Where both exist one paired
            // multiply-add per (pair, column, tap) does both; at the two ends
            // of a pair's input rows only one of them exists (scalar FMA).
            ct_u64 acc2[CT_TY / 2][CT_TX];
#pragma unroll
            for (int k = 0; k < CT_TY / 2; ++k)
#pragma unroll
                for (int tx = 0; tx < CT_TX; ++tx) acc2[k][tx] = ct_pk(0.0f, 0.0f);
#pragma unroll
            for (int r = 0; r < CT_TY + CT_FH - 1; ++r) {
                float w[CT_WWV];
                CT_LOAD_ROW(w, r);
#pragma unroll
                for (int k = 0; k < CT_TY / 2; ++k) {
                    const int i = r - 2 * k;
                    if (i >= 1 && i < CT_FH) {
#pragma unroll
                        for (int j = 0; j < CT_FW; ++j) {
                            const ct_u64 fv = p.fp[i * CT_FW + j];
#pragma unroll
                            for (int tx = 0; tx < CT_TX; ++tx)
                                acc2[k][tx] = ct_fma2(ct_pk(w[tx + j], w[tx + j]), fv, acc2[k][tx]);
                        }
                    } else if (i == 0 || i == CT_FH) {
                        const int fi = i == 0 ? 0 : CT_FH - 1;
#pragma unroll
                        for (int j = 0; j < CT_FW; ++j) {
                            const float fv = p.f[fi * CT_FW + j];
#pragma unroll
                            for (int tx = 0; tx < CT_TX; ++tx) {
                                float lo, hi;
                                ct_upk(acc2[k][tx], lo, hi);
                                if (i == 0) lo = fmaf(w[tx + j], fv, lo);
                                else hi = fmaf(w[tx + j], fv, hi);
                                acc2[k][tx] = ct_pk(lo, hi);
                            }
                        }
                    }
                }
#if CT_TY % 2
                {   // the last output row has no partner
                    const int i = r - (CT_TY - 1);
                    if (i >= 0 && i < CT_FH) {
#pragma unroll
                        for (int j = 0; j < CT_FW; ++j) {
                            const float fv = p.f[i * CT_FW + j];
#pragma unroll
                            for (int tx = 0; tx < CT_TX; ++tx)
                                acc[CT_TY - 1][tx] = fmaf(w[tx + j], fv, acc[CT_TY - 1][tx]);
                        }
                    }
                }
#endif
            }
#pragma unroll
            for (int k = 0; k < CT_TY / 2; ++k)
#pragma unroll
                for (int tx = 0; tx < CT_TX; ++tx) ct_upk(acc2[k][tx], acc[2 * k][tx], acc[2 * k + 1][tx]);
#elif CT_UNROLL == 1
            // Input row r feeds output rows ty with filter row i = r - ty.
#pragma unroll
            for (int r = 0; r < CT_TY + CT_FH - 1; ++r) {
                float w[CT_WWV];
                CT_LOAD_ROW(w, r);
#pragma unroll
                for (int ty = 0; ty < CT_TY; ++ty) {
                    const int i = r - ty;
                    if (i >= 0 && i < CT_FH) {
#pragma unroll
                        for (int j = 0; j < CT_FW; ++j) {
                            const float fv = CT_TAP(i * CT_FW + j);
#pragma unroll
                            for (int tx = 0; tx < CT_TX; ++tx)
                                acc[ty][tx] = fmaf(w[tx + j], fv, acc[ty][tx]);
                        }
                    }
                }
            }
#else
#if CT_UNROLL == 0
#pragma unroll 1
#else
#pragma unroll CT_UNROLL
#endif
            for (int i = 0; i < CT_FH; ++i) {
#pragma unroll
                for (int ty = 0; ty < CT_TY; ++ty) {
                    float w[CT_WWV];
                    CT_LOAD_ROW(w, ty + i);
#pragma unroll
                    for (int j = 0; j < CT_FW; ++j) {
                        const float fv = CT_TAP(i * CT_FW + j);
#pragma unroll
                        for (int tx = 0; tx < CT_TX; ++tx)
                            acc[ty][tx] = fmaf(w[tx + j], fv, acc[ty][tx]);
                    }
                }
            }
#endif

#pragma unroll
            for (int ty = 0; ty < CT_TY; ++ty) {
                const int y = gy + ty;
                if (y < p.out_h) {
                    float* __restrict__ orow = p.out + (ct_i64)y * p.out_pitch + gx;
#if CT_TX % 4 == 0
#pragma unroll
                    for (int k = 0; k < CT_TX; k += 4) {
                        if (gx + k + 3 < p.out_w) {
                            *reinterpret_cast<float4*>(orow + k) =
                                make_float4(acc[ty][k], acc[ty][k + 1], acc[ty][k + 2], acc[ty][k + 3]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (gx + k + e < p.out_w) orow[k + e] = acc[ty][k + e];
                        }
                    }
#else
#pragma unroll
                    for (int tx = 0; tx < CT_TX; ++tx)
                        if (gx + tx < p.out_w) orow[tx] = acc[ty][tx];
#endif
                }
            }
        }

        // next tile (persistent grid only)
        if (!p.persist) break;
        t += gridDim.x;
        if (t >= p.n_tiles) break;
        txi += p.step_x;
        tyi += p.step_y;
        if (txi >= p.tiles_x) {
            txi -= p.tiles_x;
            ++tyi;
        }
#if CT_SMEM
        // every thread is done with the staged tile (and agrees whether to go on)
        if (__syncthreads_or(!ok)) break;
#else
        if (!ok) break;
#endif
    }
#undef CT_LOAD_ROW
#undef CT_ROW_SMEM
#undef CT_TAP
}
