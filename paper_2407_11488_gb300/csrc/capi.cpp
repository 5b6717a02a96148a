// The C-ABI of libconvtune.so (declared in include/convtune.h).
#include "ct_internal.hpp"

#include <algorithm>
#include <cstdio>
#include <cstring>

using namespace ct;

extern "C" {

CT_API const char* ct_version(void) { return "convtune 0.1 (sm_103a, NVRTC variants)"; }

CT_API const char* ct_last_error(void) { return last_error(); }

CT_API ct_status ct_device_query(ct_device_info* out)
{
    if (!out) return fail(CT_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof *out);
    int n = 0, dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(CT_ERR_UNSUPPORTED, "no CUDA device is available");
    }
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    snprintf(out->name, sizeof out->name, "%.127s", prop.name);
    out->sm_count = prop.multiProcessorCount;
    out->cc_major = prop.major;
    out->cc_minor = prop.minor;
    out->smem_optin_bytes = (int32_t)prop.sharedMemPerBlockOptin;
    out->l2_bytes = prop.l2CacheSize;
    int clk = 0;
    if (cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev) != cudaSuccess) {
        cudaGetLastError();
        clk = 0;
    }
    out->clock_max_khz = clk;
    return CT_OK;
}

CT_API ct_status ct_set_cache_dir(const char* dir)
{
    cache_dir_setting() = dir ? dir : "";
    return CT_OK;
}

CT_API ct_status ct_clear_cache(void)
{
    clear_variants();
    return CT_OK;
}

CT_API ct_status ct_default_config(const ct_problem* p, ct_config* out)
{
    (void)p;
    if (!out) return fail(CT_ERR_INVALID_ARG, "out is NULL");
    *out = ct_config{32, 8, 1, 1, 0, 0};
    return CT_OK;
}

CT_API ct_status ct_check_config(const ct_problem* p, const ct_config* c, int32_t smem_limit_bytes)
{
    ct_status s = check_problem(p);
    if (s != CT_OK) return s;
    if (!c) return fail(CT_ERR_INVALID_ARG, "config is NULL");
    return check_config(*p, *c, smem_limit_bytes);
}

CT_API ct_status ct_compile(const ct_problem* p, const ct_config* c, ct_variant_info* info)
{
    return ct_compile_filter(p, c, nullptr, info);
}

CT_API ct_status ct_compile_filter(const ct_problem* p, const ct_config* c, const void* h_filter,
                                   ct_variant_info* info)
{
    ct_status s = check_problem(p);
    if (s != CT_OK) return s;
    if (!c) return fail(CT_ERR_INVALID_ARG, "config is NULL");
    if ((s = check_config(*p, *c, kDefaultSmemLimit)) != CT_OK) return s;
    VariantPtr v = get_variant(variant_key(*p, *c, h_filter));
    if (info) {
        memset(info, 0, sizeof *info);
        info->regs = v->regs;
        info->spill_bytes = v->spill_bytes;
        info->smem_bytes = (int32_t)v->smem;
        info->cubin_bytes = (int32_t)v->cubin.size();
        info->compile_ms = v->compile_ms;
        info->from_cache = v->from_cache ? 1 : 0;
    }
    if (v->status != CT_OK) return fail((ct_status)v->status, "%s", v->error.c_str());
    return CT_OK;
}

CT_API ct_status ct_device_check(int32_t clear)
{
    ct_status st = require_device();
    if (st != CT_OK) return st;
    unsigned* w = device_error_word();
    if (!w) return fail(CT_ERR_CUDA, "no device error word");
    unsigned v = 0;
    cudaError_t e = cudaMemcpy(&v, w, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read the device error word");
    if (!(v & 1u)) return CT_OK;
    if (clear && (e = cudaMemset(w, 0, 4)) != cudaSuccess) return cuda_fail(e, "clear the device error word");
    return fail(CT_ERR_TIMEOUT, "a correlation launch gave up waiting for its input copy");
}

CT_API ct_status ct_conv2d(const ct_problem* p, const ct_config* c, const void* d_image, const void* h_filter,
                           float* d_out, void* stream)
{
    ct_status s = check_problem(p);
    if (s != CT_OK) return s;
    if (!c) return fail(CT_ERR_INVALID_ARG, "config is NULL");
    if ((s = check_buffers(*p, d_image, h_filter, d_out)) != CT_OK) return s;
    if ((s = require_device()) != CT_OK) return s;
    if ((s = check_config(*p, *c, 0)) != CT_OK) return s;
    if (p->out_w == 0 || p->out_h == 0) return CT_OK;
    VariantPtr v = get_variant(variant_key(*p, *c, h_filter));
    if (v->status != CT_OK) return fail((ct_status)v->status, "%s", v->error.c_str());
    return launch_variant(*v, *p, d_image, h_filter, d_out, (cudaStream_t)stream, c->persist);
}

// Streams and events of the host-buffer pipeline, one set per device.
struct HostPipe {
    std::mutex mu;
    cudaStream_t copy_in = nullptr, copy_out = nullptr, comp[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev;
    bool ready = false;
};

static HostPipe& host_pipe(int dev)
{
    static std::mutex m;
    static auto* pipes = new std::unordered_map<int, HostPipe*>();
    std::lock_guard<std::mutex> g(m);
    HostPipe*& hp = (*pipes)[dev];
    if (!hp) hp = new HostPipe();
    return *hp;
}

static constexpr int kMaxBands = 8;

static ct_status host_pipeline(const ct_problem* p, const ct_config* c, const void* h_image, int64_t h_in_pitch,
                               const void* h_filter, float* h_out, int64_t h_out_pitch, void* d_image_ws,
                               float* d_out_ws, void* stream, cudaEvent_t done_event)
{
    ct_status s = check_problem(p);
    if (s != CT_OK) return s;
    if (!c) return fail(CT_ERR_INVALID_ARG, "config is NULL");
    if (p->out_w == 0 || p->out_h == 0) return CT_OK;
    if (!h_image || !h_out) return fail(CT_ERR_INVALID_ARG, "host image or output is NULL");
    if (h_in_pitch < in_w(*p) || h_out_pitch < p->out_w) return fail(CT_ERR_INVALID_ARG, "host pitch below the row width");
    if ((s = check_buffers(*p, d_image_ws, h_filter, d_out_ws)) != CT_OK) return s;
    if ((s = require_device()) != CT_OK) return s;
    if ((s = check_config(*p, *c, 0)) != CT_OK) return s;
    VariantPtr v = get_variant(variant_key(*p, *c, h_filter));
    if (v->status != CT_OK) return fail((ct_status)v->status, "%s", v->error.c_str());
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    HostPipe& hp = host_pipe(dev);
    std::lock_guard<std::mutex> g(hp.mu);
    if (!hp.ready) {
        cudaStream_t* all[4] = {&hp.copy_in, &hp.copy_out, &hp.comp[0], &hp.comp[1]};
        for (auto* st : all)
            if ((e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate(host pipeline)");
        hp.ev.resize(2 + 2 * kMaxBands);
        for (auto& ev : hp.ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreate(host pipeline)");
        hp.ready = true;
    }
    // Bands of output rows: band b copies in the input rows it needs that no
    // earlier band copied, runs on alternating compute streams, and copies
    // its output rows back; consecutive bands overlap copy-in, compute and
    // copy-out.
    const int64_t es = elem_size(p->dtype);
    const int bands = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxBands, p->out_h / 256));
    cudaStream_t user = (cudaStream_t)stream;
    cudaEvent_t start = hp.ev[0], done = hp.ev[1];
    cudaEventRecord(start, user);
    cudaStreamWaitEvent(hp.copy_in, start, 0);
    int64_t copied_rows = 0;
    for (int b = 0; b < bands; ++b) {
        const int64_t y0 = (int64_t)p->out_h * b / bands, y1 = (int64_t)p->out_h * (b + 1) / bands;
        const int64_t need = std::min<int64_t>(in_h(*p), y1 + p->filter_h - 1);
        cudaEvent_t e_in = hp.ev[2 + 2 * b], e_comp = hp.ev[3 + 2 * b];
        if (need > copied_rows) {
            char* dst = (char*)d_image_ws + (size_t)(copied_rows * p->in_pitch * es);
            const char* src = (const char*)h_image + (size_t)(copied_rows * h_in_pitch * es);
            if (h_in_pitch == p->in_pitch)   // same row layout: one contiguous copy
                e = cudaMemcpyAsync(dst, src, (size_t)((need - copied_rows) * p->in_pitch * es),
                                    cudaMemcpyHostToDevice, hp.copy_in);
            else
                e = cudaMemcpy2DAsync(dst, (size_t)(p->in_pitch * es), src, (size_t)(h_in_pitch * es),
                                      (size_t)(in_w(*p) * es), (size_t)(need - copied_rows), cudaMemcpyHostToDevice,
                                      hp.copy_in);
            if (e != cudaSuccess) return cuda_fail(e, "copy of an image band to the device");
            copied_rows = need;
        }
        cudaEventRecord(e_in, hp.copy_in);
        cudaStream_t cs = hp.comp[b & 1];
        cudaStreamWaitEvent(cs, e_in, 0);
        ct_problem pb = *p;
        pb.out_h = (int32_t)(y1 - y0);
        if ((s = launch_variant(*v, pb, (const char*)d_image_ws + y0 * p->in_pitch * es, h_filter,
                                d_out_ws + y0 * p->out_pitch, cs, c->persist)) != CT_OK)
            return s;
        cudaEventRecord(e_comp, cs);
        cudaStreamWaitEvent(hp.copy_out, e_comp, 0);
        if (h_out_pitch == p->out_pitch)
            e = cudaMemcpyAsync(h_out + y0 * h_out_pitch, d_out_ws + y0 * p->out_pitch,
                                (size_t)((y1 - y0) * p->out_pitch * 4), cudaMemcpyDeviceToHost, hp.copy_out);
        else
            e = cudaMemcpy2DAsync(h_out + y0 * h_out_pitch, (size_t)(h_out_pitch * 4), d_out_ws + y0 * p->out_pitch,
                                  (size_t)(p->out_pitch * 4), (size_t)p->out_w * 4, (size_t)(y1 - y0),
                                  cudaMemcpyDeviceToHost, hp.copy_out);
        if (e != cudaSuccess) return cuda_fail(e, "copy of an output band to the host");
    }
    if (done_event) {   // asynchronous form: completion is signalled on the caller's event only
        if ((e = cudaEventRecord(done_event, hp.copy_out)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        return CT_OK;
    }
    cudaEventRecord(done, hp.copy_out);
    cudaStreamWaitEvent(user, done, 0);
    if ((e = cudaStreamSynchronize(user)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return CT_OK;
}

CT_API ct_status ct_conv2d_host_pitched(const ct_problem* p, const ct_config* c, const void* h_image,
                                        int64_t h_in_pitch, const void* h_filter, float* h_out, int64_t h_out_pitch,
                                        void* d_image_ws, float* d_out_ws, void* stream)
{
    return host_pipeline(p, c, h_image, h_in_pitch, h_filter, h_out, h_out_pitch, d_image_ws, d_out_ws, stream,
                         nullptr);
}

CT_API ct_status ct_conv2d_host_async(const ct_problem* p, const ct_config* c, const void* h_image,
                                      int64_t h_in_pitch, const void* h_filter, float* h_out, int64_t h_out_pitch,
                                      void* d_image_ws, float* d_out_ws, void* stream, void* done_event)
{
    if (!done_event) return fail(CT_ERR_INVALID_ARG, "done_event is NULL");
    return host_pipeline(p, c, h_image, h_in_pitch, h_filter, h_out, h_out_pitch, d_image_ws, d_out_ws, stream,
                         (cudaEvent_t)done_event);
}

CT_API ct_status ct_conv2d_host(const ct_problem* p, const ct_config* c, const void* h_image, const void* h_filter,
                                float* h_out, void* d_image_ws, float* d_out_ws, void* stream)
{
    if (!p) return fail(CT_ERR_INVALID_ARG, "problem is NULL");
    return ct_conv2d_host_pitched(p, c, h_image, p->in_pitch, h_filter, h_out, p->out_pitch, d_image_ws, d_out_ws,
                                  stream);
}

// ---------------------------------------------------------------- spaces ---
CT_API ct_status ct_space_builtin(const char* name, ct_space** out)
{
    if (!name || !out) return fail(CT_ERR_INVALID_ARG, "name and out must be non-NULL");
    auto* s = new ct_space();
    if (!builtin_space(name, s->s)) {
        delete s;
        return fail(CT_ERR_INVALID_ARG, "unknown built-in space '%s' (small, full, paper)", name);
    }
    *out = s;
    return CT_OK;
}

CT_API ct_status ct_space_from_json(const char* json, ct_space** out)
{
    if (!json || !out) return fail(CT_ERR_INVALID_ARG, "json and out must be non-NULL");
    auto* s = new ct_space();
    std::string err;
    if (!space_from_json(json, s->s, err)) {
        delete s;
        return fail(CT_ERR_INVALID_ARG, "space JSON: %s", err.c_str());
    }
    *out = s;
    return CT_OK;
}

CT_API void ct_space_free(ct_space* s) { delete s; }

CT_API ct_status ct_space_count(const ct_space* s, const ct_problem* p, int32_t smem_limit_bytes, int64_t* n_raw,
                                int64_t* n_valid)
{
    ct_status st = check_problem(p);
    if (st != CT_OK) return st;
    if (!s) return fail(CT_ERR_INVALID_ARG, "space is NULL");
    const int lim = smem_limit_bytes > 0 ? smem_limit_bytes : device_smem_limit();
    if (n_raw) *n_raw = s->s.raw_size();
    if (n_valid) *n_valid = (int64_t)enumerate_valid(s->s, *p, lim).size();
    return CT_OK;
}

CT_API ct_status ct_space_enumerate(const ct_space* s, const ct_problem* p, int32_t smem_limit_bytes, ct_config* cfgs,
                                    int64_t* indices, int64_t cap, int64_t* n)
{
    ct_status st = check_problem(p);
    if (st != CT_OK) return st;
    if (!s) return fail(CT_ERR_INVALID_ARG, "space is NULL");
    const int lim = smem_limit_bytes > 0 ? smem_limit_bytes : device_smem_limit();
    std::vector<Entry> v = enumerate_valid(s->s, *p, lim);
    for (int64_t i = 0; i < (int64_t)v.size() && i < cap; ++i) {
        if (cfgs) cfgs[i] = v[(size_t)i].cfg;
        if (indices) indices[i] = v[(size_t)i].index;
    }
    if (n) *n = (int64_t)v.size();
    return CT_OK;
}

// ---------------------------------------------------------------- tuning ---
CT_API ct_status ct_tune(const ct_problem* p, const ct_space* s, ct_strategy st, const ct_tune_opts* opts,
                         const void* d_image, const void* h_filter, float* d_out, ct_config* best_out,
                         ct_table** table_out)
{
    return tune_gpu(p, s, st, opts, d_image, h_filter, d_out, best_out, table_out);
}

CT_API ct_status ct_tune_replay(const ct_problem* p, const ct_space* s, ct_strategy st, const ct_tune_opts* opts,
                                const double* times_ms, int64_t n_times, ct_config* best_out, ct_table** table_out)
{
    return tune_replay(p, s, st, opts, times_ms, n_times, best_out, table_out);
}

CT_API int64_t ct_table_size(const ct_table* t) { return t ? (int64_t)t->rows.size() : 0; }

CT_API ct_status ct_table_row(const ct_table* t, int64_t i, ct_row* out)
{
    if (!t || !out) return fail(CT_ERR_INVALID_ARG, "table and out must be non-NULL");
    if (i < 0 || i >= (int64_t)t->rows.size()) return fail(CT_ERR_INVALID_ARG, "row %lld out of range", (long long)i);
    *out = t->rows[(size_t)i];
    return CT_OK;
}

CT_API ct_status ct_table_info_get(const ct_table* t, ct_table_info* out)
{
    if (!t || !out) return fail(CT_ERR_INVALID_ARG, "table and out must be non-NULL");
    *out = t->info;
    return CT_OK;
}

CT_API ct_status ct_table_write(const ct_table* t, const char* path)
{
    if (!t || !path) return fail(CT_ERR_INVALID_ARG, "table and path must be non-NULL");
    return write_table(*t, path, t->tag, false);
}

CT_API void ct_table_free(ct_table* t) { delete t; }

}  // extern "C"
