// ct_batch_run_noalloc: the batched correlation for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the work
// done: code running under a memory allocator that must not grow (a serving
// process whose device memory is fully budgeted), real-time paths where an
// allocation's latency or synchronisation is not acceptable, or plugins whose
// host application owns every allocation.  The planned batch path
// (ct_batch_create) allocates its problem table, filter arena and work
// counter, and compiles a kernel at run time; this entry point instead keeps
// all of that per-call scratch in one fixed, statically allocated device array
// and uses a kernel compiled ahead of time, so a call allocates nothing.
//
// Scratch: kNoallocScratchBytes (1 MiB) of device memory, a file-scope static
// array; every GPU that loads the library holds it until the process exits.
// Layout: [work counter, 256 bytes][problem table][tile prefix sums][filters].
#include "ct_internal.hpp"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace {

constexpr size_t kNoallocScratchBytes = size_t(1) << 20;
constexpr int kNoallocMaxProblems = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// fixed tile of the ahead-of-time kernel: 32 x 8 threads, 4 x 2 outputs each
constexpr int kBX = 32, kBY = 8, kNT = kBX * kBY, kTX = 4, kTY = 2;
constexpr int kTW = kBX * kTX, kTH = kBY * kTY;
constexpr int kFmax = CT_MAX_FILTER;
constexpr int kSWmax = ((kTW + kFmax - 1) + 3) / 4 * 4;
constexpr int kHHmax = kTH + kFmax - 1;
constexpr size_t kSmemBytes = (size_t)(kFmax * kFmax + kHHmax * kSWmax) * sizeof(float);

struct NaProblem {
    const void* in;
    float* out;
    long long in_pitch, out_pitch;
    int out_w, out_h, in_w, in_h;
    int fw, fh, tiles_x, filt_off;
};
static_assert(sizeof(NaProblem) == 64, "NaProblem layout");

struct NaLayout {
    size_t problems, prefix, filters, total;
};

NaLayout layout_for(int n, size_t n_taps)
{
    NaLayout l;
    l.problems = 256;
    l.prefix = l.problems + (size_t)n * sizeof(NaProblem);
    l.filters = (l.prefix + (size_t)(n + 1) * sizeof(unsigned) + 15) / 16 * 16;
    l.total = l.filters + n_taps * sizeof(float);
    return l;
}

template <int DT>
__device__ __forceinline__ float na_load(const void* base, long long idx)
{
    if (DT == CT_F32) return __ldg(static_cast<const float*>(base) + idx);
    const unsigned short h = __ldg(static_cast<const unsigned short*>(base) + idx);
    return __uint_as_float(((unsigned)h) << 16);
}

// Persistent blocks take tiles from the counter at the start of the scratch;
// a tile's problem is found by binary search in the tile prefix sums.  Each
// output adds its taps in (i, j) order with one FMA each, as ct_conv2d does.
template <int DT>
__global__ void __launch_bounds__(kNT) noalloc_batch_kernel(unsigned char* scratch, int n, unsigned n_work,
                                                            size_t off_problems, size_t off_prefix,
                                                            size_t off_filters)
{
    extern __shared__ float na_smem[];
    __shared__ unsigned s_w;
    __shared__ int s_p;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    const NaProblem* probs = reinterpret_cast<const NaProblem*>(scratch + off_problems);
    const unsigned* prefix = reinterpret_cast<const unsigned*>(scratch + off_prefix);
    const float* filters = reinterpret_cast<const float*>(scratch + off_filters);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const unsigned w = atomicAdd(counter, 1u);
            int lo = 0, hi = n;   // last p with prefix[p] <= w
            while (hi - lo > 1) {
                const int mid = (lo + hi) / 2;
                if (prefix[mid] <= w) lo = mid;
                else hi = mid;
            }
            s_w = w;
            s_p = lo;
        }
        __syncthreads();
        const unsigned w = s_w;
        if (w >= n_work) break;
        const NaProblem pr = probs[s_p];
        const int tile = (int)(w - prefix[s_p]);
        const int gx0 = (tile % pr.tiles_x) * kTW, gy0 = (tile / pr.tiles_x) * kTH;
        const int sw = (kTW + pr.fw - 1 + 3) / 4 * 4;
        const int hh = kTH + pr.fh - 1;
        float* taps = na_smem;
        float* halo = na_smem + kFmax * kFmax;
        for (int k = tid; k < pr.fw * pr.fh; k += kNT) taps[k] = filters[pr.filt_off + k];
        for (int k = tid; k < hh * sw; k += kNT) {
            const int r = k / sw, c = k - r * sw;
            const int yy = gy0 + r, xx = gx0 + c;
            halo[k] = (yy < pr.in_h && xx < pr.in_w) ? na_load<DT>(pr.in, (long long)yy * pr.in_pitch + xx) : 0.0f;
        }
        __syncthreads();
        const int lx = (tid % kBX) * kTX, ly = (tid / kBX) * kTY;
        float acc[kTY][kTX];
#pragma unroll
        for (int ty = 0; ty < kTY; ++ty)
#pragma unroll
            for (int tx = 0; tx < kTX; ++tx) acc[ty][tx] = 0.0f;
        for (int i = 0; i < pr.fh; ++i) {
#pragma unroll
            for (int ty = 0; ty < kTY; ++ty) {
                const float* row = halo + (ly + ty + i) * sw + lx;
                float win[kTX];
#pragma unroll
                for (int tx = 0; tx < kTX; ++tx) win[tx] = row[tx];
                for (int j = 0; j < pr.fw; ++j) {
                    const float t = taps[i * pr.fw + j];
#pragma unroll
                    for (int tx = 0; tx < kTX; ++tx) acc[ty][tx] = fmaf(win[tx], t, acc[ty][tx]);
                    if (j + 1 < pr.fw) {
#pragma unroll
                        for (int tx = 0; tx < kTX - 1; ++tx) win[tx] = win[tx + 1];
                        win[kTX - 1] = row[kTX + j];
                    }
                }
            }
        }
        const int gx = gx0 + lx, gy = gy0 + ly;
#pragma unroll
        for (int ty = 0; ty < kTY; ++ty) {
            const int y = gy + ty;
            if (y < pr.out_h) {
#pragma unroll
                for (int tx = 0; tx < kTX; ++tx)
                    if (gx + tx < pr.out_w) pr.out[(long long)y * pr.out_pitch + gx + tx] = acc[ty][tx];
            }
        }
        __syncthreads();
    }
}

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};
unsigned char g_host_staging[kNoallocScratchBytes];

}  // namespace

using namespace ct;

extern "C" CT_API ct_status ct_batch_run_noalloc(const ct_batch_item* items, int32_t n, int32_t dtype, void* stream)
{
    if (!items || n <= 0) return fail(CT_ERR_INVALID_ARG, "a batch needs at least one item");
    if (n > kNoallocMaxProblems)
        return fail(CT_ERR_INVALID_ARG, "ct_batch_run_noalloc takes at most %d problems, got %d", kNoallocMaxProblems,
                    n);
    if (dtype != CT_F32 && dtype != CT_BF16) return fail(CT_ERR_INVALID_ARG, "bad dtype %d", dtype);
    size_t n_taps = 0;
    uint64_t n_work = 0;
    ct_status st;
    for (int i = 0; i < n; ++i) {
        const ct_batch_item& it = items[i];
        ct_problem p{it.out_w, it.out_h, it.filter_w, it.filter_h, it.in_pitch, it.out_pitch, dtype, 0};
        if ((st = check_problem(&p)) != CT_OK || (st = check_buffers(p, it.d_image, it.h_filter, it.d_out)) != CT_OK)
            return fail(st, "batch item %d: %s", i, last_error());
        n_taps += (size_t)it.filter_w * it.filter_h;
        if (it.out_w > 0 && it.out_h > 0)
            n_work += (uint64_t)((it.out_w + kTW - 1) / kTW) * (uint64_t)((it.out_h + kTH - 1) / kTH);
    }
    if (n_work >= 0xffffffffull) return fail(CT_ERR_INVALID_ARG, "too many tiles for ct_batch_run_noalloc");
    const NaLayout L = layout_for(n, n_taps);
    if (L.total > kNoallocScratchBytes)
        return fail(CT_ERR_INVALID_ARG,
                    "ct_batch_run_noalloc needs %zu bytes of scratch for these problems; the fixed scratch holds %zu",
                    L.total, kNoallocScratchBytes);
    if ((st = require_device()) != CT_OK) return st;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(CT_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_dev_ptr[dev]) {
        // set-up, once per device with that device current: the device
        // address of the static scratch array
        void* ptr = nullptr;
        if ((e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        const void* k32 = (const void*)noalloc_batch_kernel<CT_F32>;
        const void* k16 = (const void*)noalloc_batch_kernel<CT_BF16>;
        if ((e = cudaFuncSetAttribute(k32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(k16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes)) !=
                cudaSuccess)
            return cuda_fail(e, "cudaFuncSetAttribute(noalloc kernel)");
        g_dev_ptr[dev] = ptr;
    }
    unsigned char* dscr = static_cast<unsigned char*>(g_dev_ptr[dev]);
    // tables in the host staging area: zero counter, problems, prefix, filters
    memset(g_host_staging, 0, L.problems);
    NaProblem* probs = reinterpret_cast<NaProblem*>(g_host_staging + L.problems);
    unsigned* prefix = reinterpret_cast<unsigned*>(g_host_staging + L.prefix);
    float* taps = reinterpret_cast<float*>(g_host_staging + L.filters);
    size_t toff = 0;
    unsigned acc = 0;
    for (int i = 0; i < n; ++i) {
        const ct_batch_item& it = items[i];
        NaProblem& q = probs[i];
        q.in = it.d_image;
        q.out = it.d_out;
        q.in_pitch = it.in_pitch;
        q.out_pitch = it.out_pitch;
        q.out_w = it.out_w;
        q.out_h = it.out_h;
        q.in_w = it.out_w + it.filter_w - 1;
        q.in_h = it.out_h + it.filter_h - 1;
        q.fw = it.filter_w;
        q.fh = it.filter_h;
        q.tiles_x = (it.out_w + kTW - 1) / kTW;
        q.filt_off = (int)toff;
        const int nt = it.filter_w * it.filter_h;
        for (int k = 0; k < nt; ++k) {
            float v;
            if (dtype == CT_F32) {
                v = static_cast<const float*>(it.h_filter)[k];
            } else {
                const uint32_t u = (uint32_t) static_cast<const uint16_t*>(it.h_filter)[k] << 16;
                memcpy(&v, &u, 4);
            }
            taps[toff + (size_t)k] = v;
        }
        toff += (size_t)nt;
        prefix[i] = acc;
        if (it.out_w > 0 && it.out_h > 0)
            acc += (unsigned)(((it.out_w + kTW - 1) / kTW) * ((it.out_h + kTH - 1) / kTH));
    }
    prefix[n] = acc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemcpyAsync(dscr, g_host_staging, L.total, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(noalloc tables)");
    if (n_work == 0) return CT_OK;
    int sms = 1, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* kern = dtype == CT_F32 ? (const void*)noalloc_batch_kernel<CT_F32>
                                       : (const void*)noalloc_batch_kernel<CT_BF16>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, kSmemBytes) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)per_sm * (uint64_t)sms, n_work);
    if (dtype == CT_F32)
        noalloc_batch_kernel<CT_F32><<<grid, kNT, kSmemBytes, s>>>(dscr, n, (unsigned)n_work, L.problems, L.prefix,
                                                                   L.filters);
    else
        noalloc_batch_kernel<CT_BF16><<<grid, kNT, kSmemBytes, s>>>(dscr, n, (unsigned)n_work, L.problems, L.prefix,
                                                                    L.filters);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "launch(noalloc batch kernel)");
    return CT_OK;
}
