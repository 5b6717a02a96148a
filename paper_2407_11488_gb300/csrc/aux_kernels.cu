// Helper kernels compiled ahead of time for sm_103a: seeded scratch inputs for
// tuning runs and an L2 flush used between timed launches.
#include "ct_internal.hpp"

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Element (r, c) takes draw start + r*cols + c of SplitMix64 stream `seed`,
// mapped to (u >> 40) * 2^-23 - 1 (uniform on [-1, 1), exact in float32).
// BF16 images store that value rounded to nearest-even.
__global__ void fill_uniform_kernel(void* dst, int dtype, long long rows, long long cols, long long pitch,
                                    unsigned long long seed, unsigned long long start)
{
    const long long n = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i - r * cols;
        const unsigned long long u = mix64(seed + (start + (unsigned long long)i + 1ull) * 0x9E3779B97F4A7C15ull);
        const float v = (float)((double)(long long)(u >> 40) * 0x1p-23 - 1.0);
        if (dtype == CT_F32) {
            static_cast<float*>(dst)[r * pitch + c] = v;
        } else {
            unsigned int b = __float_as_uint(v);
            b += 0x7fffu + ((b >> 16) & 1u);
            static_cast<unsigned short*>(dst)[r * pitch + c] = (unsigned short)(b >> 16);
        }
    }
}

__global__ void l2_flush_kernel(int4* buf, long long n, unsigned int salt)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        buf[i] = make_int4((int)salt, (int)i, (int)salt, (int)i);
}

int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

namespace ct {

cudaError_t launch_fill_uniform(void* dst, int dtype, int64_t rows, int64_t cols, int64_t pitch, uint64_t seed,
                                uint64_t start, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    fill_uniform_kernel<<<grid_for(rows * cols, 256), 256, 0, s>>>(dst, dtype, rows, cols, pitch, seed, start);
    return cudaGetLastError();
}

cudaError_t launch_l2_flush(void* buf, int64_t bytes, uint32_t salt, cudaStream_t s)
{
    const long long n = bytes / 16;
    if (n <= 0) return cudaSuccess;
    l2_flush_kernel<<<grid_for(n, 512), 512, 0, s>>>(static_cast<int4*>(buf), n, salt);
    return cudaGetLastError();
}

}  // namespace ct
