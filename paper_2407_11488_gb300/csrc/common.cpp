// Errors, problem/config validation, the SplitMix64 generator and search spaces.
#include "ct_internal.hpp"

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace ct {

// ---------------------------------------------------------------- errors ---
static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }
void clear_error() { g_error.clear(); }
const char* last_error() { return g_error.c_str(); }

ct_status fail(ct_status s, const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

ct_status cuda_fail(cudaError_t e, const char* what)
{
    ct_status s = CT_ERR_CUDA;
    if (e == cudaErrorMemoryAllocation) s = CT_ERR_OOM;
    else if (e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidConfiguration) s = CT_ERR_LAUNCH;
    else if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorNoKernelImageForDevice)
        s = CT_ERR_UNSUPPORTED;
    return fail(s, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// --------------------------------------------------------------- problem ---
ct_status check_problem(const ct_problem* p)
{
    if (!p) return fail(CT_ERR_INVALID_ARG, "problem is NULL");
    if (p->dtype != CT_F32 && p->dtype != CT_BF16)
        return fail(CT_ERR_INVALID_ARG, "dtype %d is not CT_F32 or CT_BF16", p->dtype);
    if (p->filter_w < 1 || p->filter_h < 1 || p->filter_w > CT_MAX_FILTER || p->filter_h > CT_MAX_FILTER)
        return fail(CT_ERR_INVALID_ARG, "filter %dx%d outside 1..%d", p->filter_w, p->filter_h, CT_MAX_FILTER);
    if (p->out_w < 0 || p->out_h < 0)
        return fail(CT_ERR_INVALID_ARG, "negative output size %dx%d", p->out_w, p->out_h);
    if (p->in_pitch < in_w(*p))
        return fail(CT_ERR_INVALID_ARG, "in_pitch %lld < input width %lld", (long long)p->in_pitch,
                    (long long)in_w(*p));
    if (p->out_pitch < p->out_w)
        return fail(CT_ERR_INVALID_ARG, "out_pitch %lld < out_w %d", (long long)p->out_pitch, p->out_w);
    if ((p->in_pitch * elem_size(p->dtype)) % 16 != 0)
        return fail(CT_ERR_INVALID_ARG, "in_pitch %lld elements is not a multiple of 16 bytes",
                    (long long)p->in_pitch);
    if ((p->out_pitch * 4) % 16 != 0)
        return fail(CT_ERR_INVALID_ARG, "out_pitch %lld floats is not a multiple of 16 bytes",
                    (long long)p->out_pitch);
    return CT_OK;
}

int64_t smem_bytes(const ct_problem& p, const ct_config& c)
{
    if (!c.use_smem) return 0;
    const int64_t rows = (int64_t)c.block_y * c.tile_y + p.filter_h - 1;
    const int64_t cols = round_up((int64_t)c.block_x * c.tile_x + p.filter_w - 1, 4);
    return rows * cols * 4;
}

ct_status check_config(const ct_problem& p, const ct_config& c, int smem_limit)
{
    if (c.block_x < 1 || c.block_y < 1)
        return fail(CT_ERR_INVALID_CONFIG, "block %dx%d must be positive", c.block_x, c.block_y);
    if ((int64_t)c.block_x * c.block_y > kMaxThreads)
        return fail(CT_ERR_INVALID_CONFIG, "block %dx%d exceeds %d threads", c.block_x, c.block_y, kMaxThreads);
    if (c.tile_x < 1 || c.tile_y < 1 || c.tile_x > kMaxTile || c.tile_y > kMaxTile)
        return fail(CT_ERR_INVALID_CONFIG, "tile %dx%d outside 1..%d", c.tile_x, c.tile_y, kMaxTile);
    if (c.unroll != 0 && c.unroll != 1 && c.unroll != 2 && c.unroll != 4)
        return fail(CT_ERR_INVALID_CONFIG, "unroll must be 0 (rolled), 1 (full), 2 or 4 (partial factor)");
    if ((c.use_smem != 0 && c.use_smem != 1) ||
        (c.persist != 0 && c.persist != 1) || (c.taps != 0 && c.taps != 1) || (c.fma2 != 0 && c.fma2 != 1) ||
        (c.shfl != 0 && c.shfl != 1))
        return fail(CT_ERR_INVALID_CONFIG, "use_smem/persist/taps/fma2/shfl must be 0 or 1");
    if (c.use_smem && (c.block_x * c.tile_x) % 4 != 0)
        return fail(CT_ERR_INVALID_CONFIG, "use_smem needs block_x*tile_x to be a multiple of 4");
    if (smem_limit <= 0) smem_limit = device_smem_limit();
    const int64_t sb = smem_bytes(p, c);
    if (sb > smem_limit)
        return fail(CT_ERR_INVALID_CONFIG, "shared-memory tile of %lld bytes exceeds the %d-byte limit",
                    (long long)sb, smem_limit);
    return CT_OK;
}

int device_smem_limit()
{
    int dev = 0, v = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return kDefaultSmemLimit;
    }
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return kDefaultSmemLimit;
    }
    return v;
}

double problem_flops(const ct_problem& p)
{
    return 2.0 * (double)p.out_w * (double)p.out_h * (double)p.filter_w * (double)p.filter_h;
}

// ------------------------------------------------------------------ rng ----
uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- spaces ---
const char* const kParamNames[6] = {"block_x", "block_y", "tile_x", "tile_y", "use_smem", "unroll"};

int64_t Space::raw_size() const
{
    int64_t n = 1;
    for (const auto& v : vals) n *= (int64_t)v.size();
    return n;
}

ct_config Space::at(int64_t canonical) const
{
    ct_config c{};
    for (int k = 5; k >= 0; --k) {
        const int64_t m = (int64_t)vals[k].size();
        cfg_set(c, k, vals[k][canonical % m]);
        canonical /= m;
    }
    return c;
}

int64_t Space::index_of(const ct_config& c) const
{
    int64_t idx = 0;
    for (int k = 0; k < 6; ++k) {
        int pos = -1;
        for (size_t j = 0; j < vals[k].size(); ++j)
            if (vals[k][j] == cfg_get(c, k)) { pos = (int)j; break; }
        if (pos < 0) return -1;
        idx = idx * (int64_t)vals[k].size() + pos;
    }
    return idx;
}

std::vector<Entry> enumerate_valid(const Space& s, const ct_problem& p, int smem_limit)
{
    std::vector<Entry> out;
    const int64_t n = s.raw_size();
    std::string saved = last_error();
    for (int64_t i = 0; i < n; ++i) {
        ct_config c = s.at(i);
        if (check_config(p, c, smem_limit) == CT_OK) out.push_back({i, c});
    }
    set_error(saved);
    return out;
}

static std::vector<int> range_vals(int lo, int hi, int step = 1)
{
    std::vector<int> v;
    for (int x = lo; x <= hi; x += step) v.push_back(x);
    return v;
}

bool builtin_space(const char* name, Space& s)
{
    s = Space{};
    s.name = name;
    if (!strcmp(name, "small")) {
        s.vals[0] = {16, 32, 64, 128};
        s.vals[1] = {1, 2, 4, 8};
        s.vals[2] = {1, 2};
        s.vals[3] = {1, 2};
    } else if (!strcmp(name, "full")) {
        s.vals[0] = {16, 32, 64, 128, 256};
        s.vals[1] = {1, 2, 4, 8, 16};
        s.vals[2] = range_vals(1, 8);
        s.vals[3] = range_vals(1, 8);
    } else if (!strcmp(name, "paper")) {
        s.vals[0] = range_vals(16, 256, 16);
        s.vals[1] = {1, 2, 4, 8, 16};
        s.vals[2] = range_vals(1, 4);
        s.vals[3] = range_vals(1, 4);
    } else {
        return false;
    }
    s.vals[4] = {0, 1};
    s.vals[5] = {0, 1};
    return true;
}

// Minimal parser for {"name": [int, ...], ...}.
bool space_from_json(const char* js, Space& s, std::string& err)
{
    s = Space{};
    s.name = "json";
    const int defaults[6] = {32, 8, 1, 1, 0, 0};
    bool seen[6] = {false, false, false, false, false, false};
    const char* q = js;
    auto skip = [&]() { while (*q == ' ' || *q == '\n' || *q == '\t' || *q == '\r' || *q == ',') ++q; };
    skip();
    if (*q != '{') { err = "expected '{'"; return false; }
    ++q;
    for (;;) {
        skip();
        if (*q == '}') break;
        if (*q != '"') { err = "expected a quoted key"; return false; }
        const char* k0 = ++q;
        while (*q && *q != '"') ++q;
        if (!*q) { err = "unterminated key"; return false; }
        std::string key(k0, q - k0);
        ++q;
        skip();
        if (*q != ':') { err = "expected ':' after key " + key; return false; }
        ++q;
        skip();
        if (*q != '[') { err = "expected a list for " + key; return false; }
        ++q;
        std::vector<int> v;
        for (;;) {
            skip();
            if (*q == ']') { ++q; break; }
            char* end = nullptr;
            long x = strtol(q, &end, 10);
            if (end == q) { err = "expected an integer in " + key; return false; }
            v.push_back((int)x);
            q = end;
        }
        int k = -1;
        for (int j = 0; j < 6; ++j)
            if (key == kParamNames[j] || (j == 4 && key == "smem")) k = j;
        if (k < 0) { err = "unknown parameter " + key; return false; }
        if (v.empty()) { err = "empty value list for " + key; return false; }
        s.vals[k] = v;
        seen[k] = true;
    }
    for (int k = 0; k < 6; ++k)
        if (!seen[k]) s.vals[k] = {defaults[k]};
    return true;
}

}  // namespace ct
