// Variant builder: NVRTC compile of the correlation template to an sm_103a
// cubin, on-disk and in-memory caches, module loading and the launch.
#include <cuda.h>
#include <cudaTypedefs.h>
#include "ct_internal.hpp"

#include <nvrtc.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <sys/stat.h>
#include <unistd.h>

namespace ct {

// The kernel template source, embedded at build time.
static const char kCorr2dSource[] =
#include "corr2d_src.inc"
    ;

static const char* kArch = "--gpu-architecture=sm_103a";

uint64_t VariantKey::packed() const
{
    uint64_t k = 0;
    k = k * 2048 + (uint64_t)cfg.block_x;
    k = k * 2048 + (uint64_t)cfg.block_y;
    k = k * 32 + (uint64_t)cfg.tile_x;
    k = k * 32 + (uint64_t)cfg.tile_y;
    k = k * 2 + (uint64_t)cfg.use_smem;
    k = k * 8 + (uint64_t)cfg.unroll;
    k = k * 64 + (uint64_t)fw;
    k = k * 64 + (uint64_t)fh;
    k = k * 4 + (uint64_t)dtype;
    k = k * 2 + (uint64_t)(cfg.fma2 ? 1 : 0);
    k = k * 2 + (uint64_t)(cfg.shfl ? 1 : 0);
    if (!taps.empty()) {   // a filter-specific variant: mix in the taps' bits
        uint64_t h = 1469598103934665603ull;
        const unsigned char* b = reinterpret_cast<const unsigned char*>(taps.data());
        for (size_t i = 0; i < taps.size() * sizeof(float); ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
        k = (k * 0x9E3779B97F4A7C15ull) ^ h ^ 1ull;
    }
    return k;
}

VariantKey variant_key(const ct_problem& p, const ct_config& c, const void* h_filter)
{
    VariantKey k{c, p.filter_w, p.filter_h, p.dtype, {}};
    k.cfg.persist = 0;
    // paired multiply-adds: unrolled, two output rows per thread, parameter-block taps
    k.cfg.fma2 = (c.fma2 && c.unroll == 1 && c.tile_y >= 2 && !c.taps) ? 1 : 0;
    // shuffled windows: staged halo, whole warps per thread row, 4-wide register tiles
    k.cfg.shfl = (c.shfl && c.use_smem && c.block_x % 32 == 0 && c.tile_x % 4 == 0 &&
                  !(p.dtype == CT_BF16 && k.cfg.fma2)) ? 1 : 0;
    if (!(c.taps && c.unroll == 1 && h_filter) || k.cfg.fma2) {
        k.cfg.taps = 0;
        return k;
    }
    const int n = p.filter_w * p.filter_h;
    k.taps.resize((size_t)n);
    for (int i = 0; i < n; ++i) {
        float v;
        if (p.dtype == CT_F32) {
            memcpy(&v, static_cast<const float*>(h_filter) + i, 4);
        } else {
            const uint32_t u = (uint32_t) static_cast<const uint16_t*>(h_filter)[i] << 16;
            memcpy(&v, &u, 4);
        }
        if (!std::isfinite(v)) {   // no literal for it: the parameter-block form
            k.taps.clear();
            k.cfg.taps = 0;
            return k;
        }
        k.taps[(size_t)i] = v;
    }
    k.cfg.taps = 1;
    return k;
}

std::string VariantKey::describe() const
{
    char b[160];
    snprintf(b, sizeof b, "bx=%d by=%d tx=%d ty=%d smem=%d unroll=%d fw=%d fh=%d dtype=%d%s%s", cfg.block_x,
             cfg.block_y, cfg.tile_x, cfg.tile_y, cfg.use_smem, cfg.unroll, fw, fh, dtype,
             taps.empty() ? "" : " taps=compiled", cfg.fma2 ? " fma2" : cfg.shfl ? " shfl" : "");
    return b;
}

Variant::~Variant()
{
    if (lib) cudaLibraryUnload(lib);
}

std::vector<std::string> nvrtc_base_options();

// Extra NVRTC options from the environment (space separated), e.g. to inject
// a compile failure when testing how failures are recorded.
void add_env_options(std::vector<std::string>& o)
{
    if (const char* extra = getenv("CONVTUNE_NVRTC_EXTRA")) {
        std::istringstream is(extra);
        std::string tok;
        while (is >> tok) o.push_back(tok);
    }
}

static std::vector<std::string> nvrtc_options(const VariantKey& k)
{
    std::vector<std::string> o = nvrtc_base_options();
    auto def = [&](const char* n, int v) { o.push_back(std::string("-D") + n + "=" + std::to_string(v)); };
    def("CT_BX", k.cfg.block_x);
    def("CT_BY", k.cfg.block_y);
    def("CT_TX", k.cfg.tile_x);
    def("CT_TY", k.cfg.tile_y);
    def("CT_SMEM", k.cfg.use_smem);
    def("CT_UNROLL", k.cfg.unroll);
    def("CT_FW", k.fw);
    def("CT_FH", k.fh);
    def("CT_DTYPE", k.dtype);
    def("CT_TMA", tma_staged(k.cfg, k.fw, k.fh, k.dtype) ? 1 : 0);
    if (!k.taps.empty()) def("CT_TAPS_IMM", 1);
    if (k.cfg.fma2) def("CT_FMA2", 1);
    if (k.cfg.shfl) def("CT_SHFL", 1);
    add_env_options(o);
    return o;
}

// The source compiled for k: the template, preceded for a filter-specific
// variant by the taps as exact hexadecimal float literals.
static std::string variant_source(const VariantKey& k)
{
    std::string src;
    if (!k.taps.empty()) {
        src.reserve(k.taps.size() * 20 + sizeof kCorr2dSource + 64);
        src += "#define CT_TAP_VALUES ";
        char b[48];
        for (size_t i = 0; i < k.taps.size(); ++i) {
            snprintf(b, sizeof b, "%s%af", i ? ", " : "", (double)k.taps[i]);
            src += b;
        }
        src += "\n";
    }
    src.append(kCorr2dSource, sizeof kCorr2dSource - 1);
    return src;
}

int64_t halo_box_w(const ct_config& c, int fw, int dtype)
{
    return round_up((int64_t)c.block_x * c.tile_x + fw - 1, 16 / elem_size(dtype));
}
int64_t halo_box_h(const ct_config& c, int fh) { return (int64_t)c.block_y * c.tile_y + fh - 1; }
// BF16 only in the paired form: a BF16 halo copied as is is widened at every
// window load (each element is loaded by up to TY + FH - 1 rows of windows),
// which the scalar form pays from its issue slots (the per-thread staging
// widens each element once instead); the paired form leaves a third of the
// issue slots free.
bool tma_staged(const ct_config& c, int fw, int fh, int dtype)
{
    return (dtype == CT_F32 || c.fma2) && c.use_smem && halo_box_w(c, fw, dtype) <= 256 &&
           halo_box_h(c, fh) <= 256 && ((int64_t)c.block_x * c.tile_x * elem_size(dtype)) % 16 == 0;
}

unsigned* device_error_word()
{
    static std::mutex mu;
    static unsigned* words[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!words[dev]) {
        void* p = nullptr;
        if (cudaMalloc(&p, 256) != cudaSuccess || cudaMemset(p, 0, 256) != cudaSuccess) {
            cudaGetLastError();
            if (p) cudaFree(p);
            return nullptr;
        }
        words[dev] = static_cast<unsigned*>(p);
    }
    return words[dev];
}

bool take_device_error()
{
    unsigned* w = device_error_word();
    if (!w) return false;
    unsigned v = 0;
    if (cudaMemcpy(&v, w, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (v & 1u) cudaMemset(w, 0, 4);
    return (v & 1u) != 0;
}

ct_status encode_halo_map(void* map, const void* d_image, int dtype, int64_t in_w, int64_t in_h, int64_t in_pitch,
                          int64_t box_w, int64_t box_h)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        cudaGetLastError();
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return fail(CT_ERR_CUDA, "the driver offers no cuTensorMapEncodeTiled");
    const cuuint64_t dims[2] = {(cuuint64_t)in_w, (cuuint64_t)in_h};
    const cuuint64_t strides[1] = {(cuuint64_t)(in_pitch * elem_size(dtype))};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r =
        encode(static_cast<CUtensorMap*>(map),
               dtype == CT_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               const_cast<void*>(d_image), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(CT_ERR_INVALID_ARG, "cuTensorMapEncodeTiled failed (%d) for a %lldx%lld image, box %lldx%lld",
                    (int)r, (long long)in_w, (long long)in_h, (long long)box_w, (long long)box_h);
    return CT_OK;
}


static uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

static uint64_t cache_hash(const char* src, size_t len, const std::vector<std::string>& opts)
{
    int maj = 0, min = 0;
    nvrtcVersion(&maj, &min);
    uint64_t h = fnv1a(src, len);
    for (const auto& s : opts) h = fnv1a(s.c_str(), s.size() + 1, h);
    int v[2] = {maj, min};
    return fnv1a(v, sizeof v, h);
}

static void parse_ptxas(Variant& v)
{
    v.regs = 0;
    v.spill_bytes = 0;
    const char* p = strstr(v.log.c_str(), "Used ");
    if (p) v.regs = atoi(p + 5);
    const char* s = strstr(v.log.c_str(), "bytes spill stores");
    if (s) {
        const char* b = s;
        while (b > v.log.c_str() && (b[-1] == ' ' || (b[-1] >= '0' && b[-1] <= '9'))) --b;
        v.spill_bytes += atoi(b);
        const char* l = strstr(s, ", ");
        if (l) v.spill_bytes += atoi(l + 2);
    }
}

static bool read_file(const std::string& path, std::string& out)
{
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    std::stringstream ss;
    ss << f.rdbuf();
    out = ss.str();
    return true;
}

static void write_file_atomic(const std::string& path, const void* data, size_t n)
{
    std::string tmp = path + ".tmp" + std::to_string((long long)getpid()) + "_" +
                      std::to_string((unsigned long long)std::hash<std::thread::id>{}(std::this_thread::get_id()));
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    bool ok = fwrite(data, 1, n, f) == n;
    ok = (fclose(f) == 0) && ok;
    if (ok) rename(tmp.c_str(), path.c_str());
    else unlink(tmp.c_str());
}

static void mkdirs(const std::string& dir)
{
    std::string cur;
    for (size_t i = 0; i <= dir.size(); ++i) {
        if (i == dir.size() || dir[i] == '/') {
            if (!cur.empty()) mkdir(cur.c_str(), 0775);
        }
        if (i < dir.size()) cur.push_back(dir[i]);
    }
}

std::vector<std::string> nvrtc_base_options()
{
    return {kArch, "--std=c++17", "--ptxas-options=-v", "-lineinfo"};
}

VariantPtr compile_source(const char* src, size_t len, const char* prog_name, const std::vector<std::string>& opts,
                          const std::string& kernel_name, const std::string& cache_dir)
{
    auto v = std::make_shared<Variant>();
    v->kname = kernel_name;
    std::string base;
    if (!cache_dir.empty()) {
        char hex[32];
        snprintf(hex, sizeof hex, "%016llx", (unsigned long long)cache_hash(src, len, opts));
        base = cache_dir + "/ct-" + hex;
        std::string bin, log;
        if (read_file(base + ".cubin", bin) && read_file(base + ".log", log) && !bin.empty()) {
            v->cubin.assign(bin.begin(), bin.end());
            v->log = log;
            parse_ptxas(*v);
            v->from_cache = true;
            return v;
        }
    }
    const double t0 = now_ms();
    nvrtcProgram prog = nullptr;
    nvrtcResult r = nvrtcCreateProgram(&prog, src, prog_name, 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) {
        v->status = CT_ERR_COMPILE;
        v->error = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
        return v;
    }
    std::vector<const char*> co;
    for (const auto& o : opts) co.push_back(o.c_str());
    r = nvrtcCompileProgram(prog, (int)co.size(), co.data());
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string log(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &log[0]);
    while (!log.empty() && log.back() == '\0') log.pop_back();
    v->log = log;
    if (r != NVRTC_SUCCESS) {
        v->status = CT_ERR_COMPILE;
        v->error = std::string("NVRTC failed for ") + prog_name + ": " + nvrtcGetErrorString(r) + "\n" + log;
        nvrtcDestroyProgram(&prog);
        return v;
    }
    size_t cs = 0;
    nvrtcGetCUBINSize(prog, &cs);
    v->cubin.resize(cs);
    if (cs) nvrtcGetCUBIN(prog, v->cubin.data());
    nvrtcDestroyProgram(&prog);
    v->compile_ms = now_ms() - t0;
    parse_ptxas(*v);
    if (!base.empty()) {
        mkdirs(cache_dir);
        write_file_atomic(base + ".log", v->log.data(), v->log.size());
        write_file_atomic(base + ".cubin", v->cubin.data(), v->cubin.size());
    }
    return v;
}

VariantPtr compile_variant(const VariantKey& k, const std::string& cache_dir)
{
    const std::vector<std::string> opts = nvrtc_options(k);
    const std::string src = variant_source(k);
    VariantPtr v = compile_source(src.c_str(), src.size() + 1, "corr2d.cu", opts, "ct_corr2d", cache_dir);
    v->key = k;
    ct_problem p{};
    p.filter_w = k.fw;
    p.filter_h = k.fh;
    // a tensor-staged halo lands on a 128-byte boundary: 128 bytes of slack
    v->smem = tma_staged(k.cfg, k.fw, k.fh, k.dtype)
                  ? halo_box_w(k.cfg, k.fw, k.dtype) * halo_box_h(k.cfg, k.fh) * elem_size(k.dtype) + 128
                  : smem_bytes(p, k.cfg);
    if (v->status != CT_OK) v->error = "NVRTC failed for " + k.describe() + ": " + v->error;
    return v;
}

// ------------------------------------------------------- in-memory cache ---
static std::mutex g_cache_mu;
static std::unordered_map<uint64_t, VariantPtr>& cache_map()
{
    static auto* m = new std::unordered_map<uint64_t, VariantPtr>();
    return *m;
}
static std::unordered_map<uint64_t, std::shared_future<VariantPtr>>& pending_map()
{
    static auto* m = new std::unordered_map<uint64_t, std::shared_future<VariantPtr>>();
    return *m;
}

std::string& cache_dir_setting()
{
    static std::string* dir = [] {
        const char* e = getenv("CONVTUNE_CACHE_DIR");
        return new std::string(e ? e : "");
    }();
    return *dir;
}

VariantPtr get_variant(const VariantKey& k)
{
    const uint64_t key = k.packed();
    std::shared_ptr<std::promise<VariantPtr>> mine;
    std::shared_future<VariantPtr> fut;
    std::string dir;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto it = cache_map().find(key);
        if (it != cache_map().end()) return it->second;
        auto pit = pending_map().find(key);
        if (pit != pending_map().end()) {
            fut = pit->second;
        } else {
            mine = std::make_shared<std::promise<VariantPtr>>();
            fut = mine->get_future().share();
            pending_map()[key] = fut;
            dir = cache_dir_setting();
        }
    }
    if (mine) {
        VariantPtr v = compile_variant(k, dir);
        {
            std::lock_guard<std::mutex> g(g_cache_mu);
            if (v->status == CT_OK) cache_map()[key] = v;
            pending_map().erase(key);
        }
        mine->set_value(v);
        return v;
    }
    return fut.get();
}

void put_variant(const VariantPtr& v)
{
    if (!v || v->status != CT_OK) return;
    std::lock_guard<std::mutex> g(g_cache_mu);
    cache_map()[v->key.packed()] = v;
}

void clear_variants()
{
    std::lock_guard<std::mutex> g(g_cache_mu);
    cache_map().clear();
}

// ------------------------------------------------------------- loading ----
ct_status require_device()
{
    int dev = -1, n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(CT_ERR_UNSUPPORTED, "no CUDA device is available (%s)",
                    e == cudaSuccess ? "0 devices" : cudaGetErrorString(e));
    }
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int maj = 0, min = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
    if (maj != 10 || min != 3)
        return fail(CT_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library targets sm_103a (GB300) only", dev,
                    maj, min);
    return CT_OK;
}

ct_status load_variant(Variant& v)
{
    if (v.status != CT_OK) return fail((ct_status)v.status, "%s", v.error.c_str());
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> g(v.mu);
    if (!v.lib) {
        e = cudaLibraryLoadData(&v.lib, v.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e != cudaSuccess) {
            v.lib = nullptr;
            return cuda_fail(e, "cudaLibraryLoadData");
        }
        e = cudaLibraryGetKernel(&v.kern, v.lib, v.kname.c_str());
        if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryGetKernel");
        if (v.regs == 0) {   // no ptxas report (e.g. a compile NVRTC served itself): ask the driver
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, (const void*)v.kern) == cudaSuccess) v.regs = fa.numRegs;
            else cudaGetLastError();
        }
    }
    if (v.loaded_device != dev || v.smem_attr != v.smem) {
        e = cudaFuncSetAttribute((const void*)v.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)v.kern,
                                                          v.key.cfg.block_x * v.key.cfg.block_y,
                                                          (size_t)v.smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            per_sm = sms = 0;
        }
        v.resident = std::max(0, per_sm) * std::max(0, sms);
        v.loaded_device = dev;
        v.smem_attr = v.smem;
    }
    return CT_OK;
}

void unload_variant(Variant& v)
{
    std::lock_guard<std::mutex> g(v.mu);
    if (v.lib) cudaLibraryUnload(v.lib);
    v.lib = nullptr;
    v.kern = nullptr;
    v.loaded_device = -1;
    v.smem_attr = -1;
    v.resident = 0;
}

// -------------------------------------------------------------- launch ----
ct_status check_buffers(const ct_problem& p, const void* d_image, const void* h_filter, const float* d_out)
{
    if (!h_filter) return fail(CT_ERR_INVALID_ARG, "filter pointer is NULL");
    if (p.out_w == 0 || p.out_h == 0) return CT_OK;
    if (!d_image || !d_out) return fail(CT_ERR_INVALID_ARG, "image or output pointer is NULL");
    if (((uintptr_t)d_image & 15) || ((uintptr_t)d_out & 15))
        return fail(CT_ERR_INVALID_ARG, "image and output must be 16-byte aligned");
    return CT_OK;
}

// Parameter block of ct_corr2d, laid out as the device struct CtParams: the
// image's tensor map (128 bytes, 64-byte aligned; zero for variants that do
// not use it), in, out, in_pitch, out_pitch (8 bytes each), out_w, out_h,
// in_w, in_h (4 bytes each), the error word's address (8 bytes), tiles_x,
// n_tiles, persist, step_x, step_y and one spare (4 bytes each), then
// filter_h*filter_w floats, then (paired multiply-add variants) at the next
// 8-byte boundary filter_h*filter_w tap pairs of 8 bytes; the struct's size
// is a multiple of 64 bytes.
static constexpr size_t kParamHeader = 208;
static constexpr size_t kParamMax =
    (kParamHeader + 4 * CT_MAX_FILTER * CT_MAX_FILTER + 8 + 8 * CT_MAX_FILTER * CT_MAX_FILTER + 63) / 64 * 64;

int64_t tile_count(const ct_problem& p, const ct_config& c)
{
    const int64_t tw = (int64_t)c.block_x * c.tile_x, th = (int64_t)c.block_y * c.tile_y;
    return ((p.out_w + tw - 1) / tw) * ((p.out_h + th - 1) / th);
}

ct_status launch_variant(Variant& v, const ct_problem& p, const void* d_image, const void* h_filter,
                         float* d_out, cudaStream_t stream, int persist)
{
    if (p.out_w == 0 || p.out_h == 0) return CT_OK;
    ct_status s = load_variant(v);
    if (s != CT_OK) return s;
    const ct_config& c = v.key.cfg;
    const int64_t tw = (int64_t)c.block_x * c.tile_x, th = (int64_t)c.block_y * c.tile_y;
    const int64_t gx = (p.out_w + tw - 1) / tw, gy = (p.out_h + th - 1) / th;
    if (gx > 0x7fffffffLL || gy > 65535 || gx * gy > 0x7fffffffLL)
        return fail(CT_ERR_INVALID_ARG, "grid %lldx%lld exceeds the launch limits for this config", (long long)gx,
                    (long long)gy);
    const int64_t n_tiles = gx * gy;
    // the persistent grid: the blocks the GPU holds at once (never more than the tiles)
    const int64_t g1 = persist ? std::min<int64_t>(n_tiles, std::max(1, v.resident)) : 0;
    const int32_t tiling[6] = {(int32_t)gx, (int32_t)n_tiles, persist ? 1 : 0, (int32_t)(g1 % gx),
                               (int32_t)(g1 / gx), 0};
    const int nt = p.filter_w * p.filter_h;
    alignas(64) unsigned char buf[kParamMax];
    memset(buf, 0, kTensorMapBytes);
    if (tma_staged(c, p.filter_w, p.filter_h, p.dtype)) {
        s = encode_halo_map(buf, d_image, p.dtype, in_w(p), in_h(p), p.in_pitch, halo_box_w(c, p.filter_w, p.dtype),
                            halo_box_h(c, p.filter_h));
        if (s != CT_OK) return s;
    }
    unsigned* err = device_error_word();
    if (!err) return fail(CT_ERR_CUDA, "no device error word");
    const void* in_ptr = d_image;
    void* out_ptr = d_out;
    const int64_t ipitch = p.in_pitch, opitch = p.out_pitch;
    const int32_t dims[4] = {p.out_w, p.out_h, (int32_t)in_w(p), (int32_t)in_h(p)};
    memcpy(buf + 128, &in_ptr, 8);
    memcpy(buf + 136, &out_ptr, 8);
    memcpy(buf + 144, &ipitch, 8);
    memcpy(buf + 152, &opitch, 8);
    memcpy(buf + 160, dims, 16);
    memcpy(buf + 176, &err, 8);
    memcpy(buf + 184, tiling, sizeof tiling);
    float* taps = reinterpret_cast<float*>(buf + kParamHeader);
    if (p.dtype == CT_F32) {
        memcpy(taps, h_filter, 4 * (size_t)nt);
    } else {
        const uint16_t* hb = (const uint16_t*)h_filter;
        for (int i = 0; i < nt; ++i) {
            uint32_t u = (uint32_t)hb[i] << 16;
            memcpy(&taps[i], &u, 4);
        }
    }
    if (v.key.cfg.fma2) {   // tap pairs (f[i][j], f[i-1][j]) for i >= 1
        unsigned char* fp = buf + round_up((int64_t)(kParamHeader + 4 * (size_t)nt), 8);
        memset(fp, 0, 8 * (size_t)p.filter_w);   // row 0 has no pair
        for (int i = 1; i < p.filter_h; ++i)
            for (int j = 0; j < p.filter_w; ++j) {
                memcpy(fp + 8 * (size_t)(i * p.filter_w + j), &taps[i * p.filter_w + j], 4);
                memcpy(fp + 8 * (size_t)(i * p.filter_w + j) + 4, &taps[(i - 1) * p.filter_w + j], 4);
            }
    }
    void* args[1] = {buf};
    const dim3 grid = persist ? dim3((unsigned)g1, 1, 1) : dim3((unsigned)gx, (unsigned)gy, 1);
    cudaError_t e = cudaLaunchKernel((const void*)v.kern, grid, dim3((unsigned)c.block_x, (unsigned)c.block_y, 1),
                                     args, (size_t)v.smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernel(ct_corr2d)");
    return CT_OK;
}

}  // namespace ct
