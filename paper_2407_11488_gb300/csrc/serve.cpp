// Request server: continuous batching of correlation requests onto the
// persistent batch kernel, with admission by a device-memory budget.
//
// A dispatcher thread moves each request through
//   pending -> admitted (device memory reserved from the budget, image copy
//   queued) -> ready (copy landed) -> running (in a launch) -> done (output
//   copied back, memory returned).
// Ready requests are gathered into one persistent-kernel launch; up to
// `max_launches` launches run at once on separate streams, so requests that
// arrive while others are on the GPU start as soon as memory and a launch slot
// are free, and their work overlaps with the running launches.  Each filter
// size has one tile configuration (tuned at creation, then resident), so a
// request's result does not depend on what it was batched with.  No device
// code waits on anything: the host observes completion through events.
#include "batch_internal.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

using namespace ct;

namespace {

// First-fit allocator over one device arena (offsets, 256-byte granules).
class Arena {
public:
    void init(size_t size)
    {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t n, size_t& off)
    {
        n = (n + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used_ += n;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) / 256 * 256;
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

enum class RState { Pending, Admitted, Ready, Running, Done, Failed };

struct Request {
    uint64_t id = 0;
    ct_request rq{};
    std::vector<float> taps;          // FP32, rows padded to 4 taps
    int bucket = 0;
    RState state = RState::Pending;
    size_t img_off = 0, img_bytes = 0, out_off = 0, out_bytes = 0;
    bool own_image = true;
    const void* d_image = nullptr;
    int64_t in_pitch = 0;             // device image pitch (elements)
    int64_t out_dpitch = 0;           // device output pitch (floats)
    cudaEvent_t ev_in = nullptr;
    double t_submit = 0, t_ready = 0, t_done = 0;
    int status = CT_OK;
};

struct Image {
    size_t off = 0, bytes = 0;
    int32_t in_w = 0, in_h = 0;
    int64_t in_pitch = 0;
    int users = 0;
};

struct Launch {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t k0 = nullptr, k1 = nullptr;   // around the kernel (timing events)
    bool busy = false;
    std::vector<std::shared_ptr<Request>> reqs;
    size_t tab_off = 0, tab_bytes = 0;
    unsigned char* staging = nullptr;
    size_t staging_bytes = 0;
    ct_status launched = CT_OK;   // status of starting the kernel
};

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ct_server {
    ct_server_opts o{};
    int device = 0;
    int threads = 256;
    std::vector<BucketDesc> buckets;
    VariantPtr module;
    int max_grid = 1;
    unsigned char* base = nullptr;   // device arena
    Arena arena;
    cudaStream_t copy_in = nullptr;
    std::vector<Launch> launches;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending, admitted, ready;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    std::unordered_map<uint64_t, Image> images;
    uint64_t next_id = 1, next_image = 1;
    bool stop = false;
    std::thread worker;
    // statistics since the last reset
    cudaEvent_t ref = nullptr;                      // recorded at the reset: origin of kernel intervals
    std::vector<std::pair<float, float>> kbusy;     // kernel intervals (ms after ref)
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, failed = 0, n_launches = 0, launched_reqs = 0;
    double flops = 0, t0 = 0, t_last = 0;
    int fatal = CT_OK;
    std::string fatal_msg;

    ~ct_server();
    void loop();
    int bucket_of(int fw, int fh) const
    {
        for (size_t k = 0; k < buckets.size(); ++k)
            if (buckets[k].fw == fw && buckets[k].fh == fh) return (int)k;
        return -1;
    }
    bool step_locked();
    bool launch_locked(Launch& L);
};

ct_server::~ct_server()
{
    {
        std::lock_guard<std::mutex> g(mu);
        stop = true;
    }
    cv_work.notify_all();
    if (worker.joinable()) worker.join();
    cudaSetDevice(device);
    for (auto& L : launches) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.done) cudaEventDestroy(L.done);
        if (L.k0) cudaEventDestroy(L.k0);
        if (L.k1) cudaEventDestroy(L.k1);
        if (L.staging) cudaFreeHost(L.staging);
    }
    if (ref) cudaEventDestroy(ref);
    if (copy_in) {
        cudaStreamSynchronize(copy_in);
        cudaStreamDestroy(copy_in);
    }
    for (auto& kv : reqs)
        if (kv.second->ev_in) cudaEventDestroy(kv.second->ev_in);
    if (base) cudaFree(base);
}

// One pass of the dispatcher; returns true when it changed something.
bool ct_server::step_locked()
{
    bool progress = false;
    // completions
    for (auto& L : launches) {
        if (!L.busy) continue;
        const cudaError_t e = cudaEventQuery(L.done);
        if (e == cudaErrorNotReady) continue;
        const double t = now_s();
        unsigned kerr = 0;
        memcpy(&kerr, L.staging + 4, 4);
        const bool good = e == cudaSuccess && kerr == 0 && L.launched == CT_OK;
        const ct_status why = e != cudaSuccess ? CT_ERR_CUDA : (L.launched != CT_OK ? L.launched : CT_ERR_TIMEOUT);
        for (auto& r : L.reqs) {
            r->state = good ? RState::Done : RState::Failed;
            r->status = good ? CT_OK : why;
            r->t_done = t;
            if (r->own_image) arena.release(r->img_off, r->img_bytes);
            else images[r->rq.image_id].users--;
            arena.release(r->out_off, r->out_bytes);
            if (good) {
                lat_ms.push_back(1e3 * (t - r->t_submit));
                completed++;
                flops += 2.0 * r->rq.out_w * (double)r->rq.out_h * r->rq.filter_w * r->rq.filter_h;
            } else {
                failed++;
            }
        }
        if (e != cudaSuccess) {
            fatal = CT_ERR_CUDA;
            fatal_msg = std::string("batch launch failed: ") + cudaGetErrorString(e);
        } else if (L.launched == CT_OK) {
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, ref, L.k0) == cudaSuccess && cudaEventElapsedTime(&b, ref, L.k1) == cudaSuccess)
                kbusy.emplace_back(a, b);
            else
                cudaGetLastError();
        }
        arena.release(L.tab_off, L.tab_bytes);
        L.reqs.clear();
        L.busy = false;
        t_last = t;
        progress = true;
        cv_done.notify_all();
    }
    // admission in arrival order, while the budget has room
    while (!pending.empty()) {
        auto& r = pending.front();
        size_t img_off = 0, out_off = 0;
        const size_t out_bytes = (size_t)r->rq.out_h * (size_t)r->out_dpitch * 4;
        if (!arena.alloc(std::max<size_t>(out_bytes, 256), out_off)) break;
        if (r->own_image) {
            if (!arena.alloc(std::max<size_t>(r->img_bytes, 256), img_off)) {
                arena.release(out_off, std::max<size_t>(out_bytes, 256));
                break;
            }
        }
        r->out_off = out_off;
        r->out_bytes = std::max<size_t>(out_bytes, 256);
        if (r->own_image) {
            r->img_off = img_off;
            r->img_bytes = std::max<size_t>(r->img_bytes, 256);
            r->d_image = base + img_off;
            const size_t es = (size_t)elem_size(o.dtype);
            cudaMemcpy2DAsync(base + img_off, (size_t)r->in_pitch * es, r->rq.h_image, (size_t)r->rq.in_pitch * es,
                              (size_t)(r->rq.out_w + r->rq.filter_w - 1) * es,
                              (size_t)(r->rq.out_h + r->rq.filter_h - 1), cudaMemcpyHostToDevice, copy_in);
        }
        cudaEventRecord(r->ev_in, copy_in);
        r->state = RState::Admitted;
        admitted.push_back(r);
        pending.pop_front();
        progress = true;
    }
    // copies that have landed
    while (!admitted.empty()) {
        const cudaError_t e = cudaEventQuery(admitted.front()->ev_in);
        if (e == cudaErrorNotReady) break;
        admitted.front()->state = RState::Ready;
        admitted.front()->t_ready = now_s();
        ready.push_back(admitted.front());
        admitted.pop_front();
        progress = true;
    }
    // launches: now if the GPU has nothing of ours, else when a batch is full
    // or its oldest request has waited max_wait_us
    int busy = 0;
    for (auto& L : launches) busy += L.busy ? 1 : 0;
    for (auto& L : launches) {
        if (ready.empty() || L.busy) continue;
        const bool full = (int)ready.size() >= o.max_batch;
        const bool aged = now_s() - ready.front()->t_ready >= o.max_wait_us * 1e-6;
        if (!(busy == 0 || full || aged)) break;
        if (!launch_locked(L)) break;
        busy++;
        progress = true;
    }
    return progress;
}

bool ct_server::launch_locked(Launch& L)
{
    // take ready requests while their tables fit the staging buffer
    std::vector<std::shared_ptr<Request>> take;
    size_t n_taps = 0;
    int64_t n_work = 0;
    auto tiles = [&](const Request& r, int64_t* tx) {
        const TileCfg& c = buckets[(size_t)r.bucket].cfg;
        const int64_t tw = tile_w(threads, c), th = tile_h(threads, c);
        const int64_t a = (r.rq.out_w + tw - 1) / tw, b = (r.rq.out_h + th - 1) / th;
        if (tx) *tx = a;
        return a * b;
    };
    auto bytes_for = [&](size_t np, size_t nt, int64_t nw) {
        return 256 + np * (kTensorMapBytes + sizeof(DevProblem)) + ((nt * 4 + 255) / 256) * 256 +
               (size_t)nw * sizeof(WorkItem) + 256;
    };
    while (!ready.empty() && (int)take.size() < o.max_batch) {
        const Request& r = *ready.front();
        const int64_t nt = tiles(r, nullptr);
        if (!take.empty() && bytes_for(take.size() + 1, n_taps + r.taps.size(), n_work + nt) > L.staging_bytes) break;
        if (n_work + nt > 0x7fffffffLL) break;
        n_taps += r.taps.size();
        n_work += nt;
        take.push_back(ready.front());
        ready.pop_front();
    }
    if (take.empty()) return false;
    size_t tab_bytes = bytes_for(take.size(), n_taps, n_work);
    if (tab_bytes > L.staging_bytes) {   // a single request larger than the staging buffer
        for (auto& r : take) {
            r->state = RState::Failed;
            r->status = CT_ERR_UNSUPPORTED;
            failed++;
        }
        cv_done.notify_all();
        return true;
    }
    size_t tab_off = 0;
    if (!arena.alloc(tab_bytes, tab_off)) {
        for (auto it = take.rbegin(); it != take.rend(); ++it) ready.push_front(*it);
        return false;
    }
    // host tables: [counter and error word, 256][tensor maps][problems][filters][work]
    unsigned char* st = L.staging;
    memset(st, 0, 256);
    unsigned char* maps = st + 256;
    const size_t off_p = 256 + take.size() * kTensorMapBytes;
    DevProblem* probs = reinterpret_cast<DevProblem*>(st + off_p);
    const size_t off_f = off_p + take.size() * sizeof(DevProblem);
    float* filt = reinterpret_cast<float*>(st + off_f);
    const size_t off_w = off_f + ((n_taps * 4 + 255) / 256) * 256;
    WorkItem* work = reinterpret_cast<WorkItem*>(st + off_w);
    size_t toff = 0;
    int64_t w = 0;
    for (size_t i = 0; i < take.size(); ++i) {
        const Request& r = *take[i];
        int64_t tx = 0;
        const int64_t nt = tiles(r, &tx);
        DevProblem& d = probs[i];
        d.in = r.d_image;
        d.out = reinterpret_cast<float*>(base + r.out_off);
        d.in_pitch = r.in_pitch;
        d.out_pitch = r.out_dpitch;
        d.out_w = r.rq.out_w;
        d.out_h = r.rq.out_h;
        d.in_w = r.rq.out_w + r.rq.filter_w - 1;
        d.in_h = r.rq.out_h + r.rq.filter_h - 1;
        d.bucket = r.bucket;
        d.tiles_x = (int32_t)tx;
        d.filt_off = (int32_t)toff;
        d.pad = 0;
        const TileCfg& c = buckets[(size_t)r.bucket].cfg;
        const ct_status ms = encode_halo_map(maps + i * kTensorMapBytes, r.d_image, o.dtype, d.in_w, d.in_h,
                                             r.in_pitch, batch_box_w(threads, c, r.rq.filter_w, o.dtype),
                                             batch_box_h(threads, c, r.rq.filter_h));
        if (ms != CT_OK) {
            fatal = ms;
            fatal_msg = last_error();
        }
        memcpy(filt + toff, r.taps.data(), r.taps.size() * 4);
        toff += r.taps.size();
        for (int64_t k = 0; k < nt; ++k) work[w++] = work_item((uint32_t)i, k, tx, d.bucket, d.filt_off);
    }
    unsigned char* dt = base + tab_off;
    cudaMemcpyAsync(dt, st, tab_bytes, cudaMemcpyHostToDevice, L.stream);
    DevParams prm{dt + off_p, dt + off_w, reinterpret_cast<const float*>(dt + off_f), dt + 256,
                  reinterpret_cast<unsigned*>(dt), (int32_t)n_work, 0};
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(max_grid, n_work));
    cudaEventRecord(L.k0, L.stream);
    ct_status s = fatal == CT_OK ? launch_batch(*module, grid, threads, prm, L.stream) : (ct_status)fatal;
    cudaEventRecord(L.k1, L.stream);
    if (s != CT_OK && fatal == CT_OK) {
        fatal = s;
        fatal_msg = last_error();
    }
    L.launched = s;
    // the kernel's error word comes back into the (already uploaded) staging buffer
    cudaMemcpyAsync(L.staging + 4, dt + 4, 4, cudaMemcpyDeviceToHost, L.stream);
    for (auto& r : take) {
        cudaMemcpy2DAsync((void*)r->rq.h_out, (size_t)r->rq.out_pitch * 4, base + r->out_off,
                          (size_t)r->out_dpitch * 4, (size_t)r->rq.out_w * 4, (size_t)r->rq.out_h,
                          cudaMemcpyDeviceToHost, L.stream);
        r->state = RState::Running;
    }
    cudaEventRecord(L.done, L.stream);
    L.reqs = std::move(take);
    L.tab_off = tab_off;
    L.tab_bytes = tab_bytes;
    L.busy = true;
    n_launches++;
    launched_reqs += (int64_t)L.reqs.size();
    return true;
}

void ct_server::loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> g(mu);
    for (;;) {
        const bool progress = step_locked();
        bool any = !pending.empty() || !admitted.empty() || !ready.empty();
        for (auto& L : launches) any = any || L.busy;
        if (stop && !any) return;
        if (!progress) {
            // bounded wait: new submissions wake us, device progress is polled
            cv_work.wait_for(g, std::chrono::microseconds(any ? 20 : 2000));
        }
    }
}

extern "C" {

CT_API ct_status ct_server_create(const ct_server_opts* opts, ct_server** out)
{
    if (!opts || !out) return fail(CT_ERR_INVALID_ARG, "opts and out must be non-NULL");
    *out = nullptr;
    ct_server_opts o = *opts;
    if (o.dtype != CT_F32 && o.dtype != CT_BF16) return fail(CT_ERR_INVALID_ARG, "bad dtype %d", o.dtype);
    if (o.mem_budget_bytes <= 0) return fail(CT_ERR_INVALID_ARG, "mem_budget_bytes must be positive");
    if (o.max_batch <= 0) o.max_batch = 64;
    if (o.max_launches <= 0) o.max_launches = 3;
    if (o.max_wait_us <= 0) o.max_wait_us = 200;
    if (o.filter_min <= 0) o.filter_min = 3;
    if (o.filter_max <= 0) o.filter_max = 17;
    if (o.filter_min > o.filter_max || o.filter_max > CT_MAX_FILTER)
        return fail(CT_ERR_INVALID_ARG, "filter range %d..%d invalid", o.filter_min, o.filter_max);
    if (o.staging_bytes <= 0) o.staging_bytes = 16 << 20;
    ct_status st = require_device();
    if (st != CT_OK) return st;
    auto S = std::unique_ptr<ct_server>(new ct_server());
    S->o = o;
    S->threads = 256;
    cudaGetDevice(&S->device);
    // one bucket per square filter size of the range's parity (odd range: odd sizes)
    std::vector<int> sizes;
    for (int f = o.filter_min; f <= o.filter_max; f += (o.filter_min % 2) ? 2 : 1) sizes.push_back(f);
    if (sizes.size() > 16) return fail(CT_ERR_UNSUPPORTED, "more than 16 filter sizes");
    for (int f : sizes) S->buckets.push_back(BucketDesc{f, f, TileCfg{32, 4, 2, 1}});
    if (o.tune) {
        // the tuner of ct_batch_create on representative problems per size
        cudaError_t e;
        std::vector<void*> bufs;
        std::vector<ct_batch_item> items;
        std::vector<std::vector<float>> hf;
        const int sides[3] = {160, 640, 1600};
        for (int f : sizes)
            for (int side : sides) {
                const int64_t ip = round_up(side + f - 1, 8), op = round_up(side, 4);
                void *di = nullptr, *dout = nullptr;
                if ((e = cudaMalloc(&di, (size_t)(side + f - 1) * ip * elem_size(o.dtype))) != cudaSuccess ||
                    (e = cudaMalloc(&dout, (size_t)side * op * 4)) != cudaSuccess) {
                    for (void* b : bufs) cudaFree(b);
                    if (di) cudaFree(di);
                    return cuda_fail(e, "cudaMalloc(server tuning)");
                }
                bufs.push_back(di);
                bufs.push_back(dout);
                launch_fill_uniform(di, o.dtype, side + f - 1, side + f - 1, ip, 77, 0, nullptr);
                hf.emplace_back((size_t)f * f, 0.25f);
                items.push_back(ct_batch_item{di, (float*)dout, hf.back().data(), side, side, f, f, ip, op});
            }
        cudaDeviceSynchronize();
        ct_batch_opts bo{};
        bo.dtype = o.dtype;
        bo.tune = 1;
        bo.side_split = -1;
        bo.solo_wave_pct = -1;   // every representative problem tunes its bucket
        // scalar tiles only: requests bring their taps in the plain row layout,
        // and the served launches are bound by host work, not by the FMA pipe
        bo.bucket_forms = 1;
        ct_batch* tb = nullptr;
        st = ct_batch_create(items.data(), (int32_t)items.size(), &bo, &tb);
        if (st == CT_OK) {
            for (auto& d : S->buckets) {
                for (int k = 0; k < 16; ++k) {
                    int32_t fw = 0, fh = 0, n = 0;
                    ct_bucket_config c{};
                    if (ct_batch_bucket(tb, k, &fw, &fh, &n, &c, nullptr) != CT_OK) break;
                    if (fw == d.fw && fh == d.fh) d.cfg = TileCfg{c.block_x, c.tile_x, c.tile_y, c.unroll};
                }
            }
            ct_batch_free(tb);
        }
        for (void* b : bufs) cudaFree(b);
        if (st != CT_OK) return st;
    }
    S->module = compile_batch(S->threads, o.dtype, S->buckets, cache_dir_setting());
    if (S->module->status != CT_OK) return fail(CT_ERR_COMPILE, "%s", S->module->error.c_str());
    if ((st = load_variant(*S->module)) != CT_OK) return st;
    S->max_grid = occupancy_grid(*S->module, S->threads, 0, 1 << 30);
    cudaError_t e;
    if ((e = cudaMalloc((void**)&S->base, (size_t)o.mem_budget_bytes)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(server memory budget)");
    S->arena.init((size_t)o.mem_budget_bytes);
    if ((e = cudaStreamCreateWithFlags(&S->copy_in, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    S->launches.resize((size_t)o.max_launches);
    for (auto& L : S->launches) {
        if ((e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreate(&L.k0)) != cudaSuccess || (e = cudaEventCreate(&L.k1)) != cudaSuccess ||
            (e = cudaMallocHost((void**)&L.staging, (size_t)o.staging_bytes)) != cudaSuccess)
            return cuda_fail(e, "server launch slot");
        L.staging_bytes = (size_t)o.staging_bytes;
    }
    if ((e = cudaEventCreate(&S->ref)) != cudaSuccess || (e = cudaEventRecord(S->ref, S->copy_in)) != cudaSuccess)
        return cuda_fail(e, "server reference event");
    S->t0 = S->t_last = now_s();
    ct_server* raw = S.get();
    S->worker = std::thread([raw] { raw->loop(); });
    *out = S.release();
    return CT_OK;
}

CT_API ct_status ct_server_image_register(ct_server* s, const void* h_image, int32_t in_w, int32_t in_h,
                                          int64_t in_pitch, uint64_t* image_id)
{
    if (!s || !h_image || !image_id) return fail(CT_ERR_INVALID_ARG, "NULL argument");
    if (in_w <= 0 || in_h <= 0 || in_pitch < in_w || (in_pitch * elem_size(s->o.dtype)) % 16)
        return fail(CT_ERR_INVALID_ARG, "bad image geometry");
    const size_t bytes = (size_t)in_h * (size_t)in_pitch * (size_t)elem_size(s->o.dtype);
    std::unique_lock<std::mutex> g(s->mu);
    size_t off = 0;
    if (!s->arena.alloc(bytes, off)) return fail(CT_ERR_OOM, "image does not fit the memory budget now");
    cudaError_t e = cudaMemcpy(s->base + off, h_image, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        s->arena.release(off, bytes);
        return cuda_fail(e, "upload resident image");
    }
    Image im;
    im.off = off;
    im.bytes = bytes;
    im.in_w = in_w;
    im.in_h = in_h;
    im.in_pitch = in_pitch;
    *image_id = s->next_image++;
    s->images[*image_id] = im;
    return CT_OK;
}

CT_API ct_status ct_server_image_release(ct_server* s, uint64_t image_id)
{
    if (!s) return fail(CT_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> g(s->mu);
    auto it = s->images.find(image_id);
    if (it == s->images.end()) return fail(CT_ERR_INVALID_ARG, "unknown image %llu", (unsigned long long)image_id);
    if (it->second.users > 0) return fail(CT_ERR_INVALID_ARG, "image still used by queued requests");
    s->arena.release(it->second.off, it->second.bytes);
    s->images.erase(it);
    return CT_OK;
}

CT_API ct_status ct_server_submit(ct_server* s, const ct_request* rq, uint64_t* request_id)
{
    if (!s || !rq || !request_id) return fail(CT_ERR_INVALID_ARG, "NULL argument");
    if (!rq->h_out || !rq->h_filter) return fail(CT_ERR_INVALID_ARG, "h_out and h_filter are required");
    const int b = s->bucket_of(rq->filter_w, rq->filter_h);
    if (b < 0)
        return fail(CT_ERR_UNSUPPORTED, "filter %dx%d is not served (square sizes %d..%d)", rq->filter_w,
                    rq->filter_h, s->o.filter_min, s->o.filter_max);
    if (rq->out_w <= 0 || rq->out_h <= 0) return fail(CT_ERR_INVALID_ARG, "empty request");
    if (rq->out_pitch < rq->out_w) return fail(CT_ERR_INVALID_ARG, "out_pitch < out_w");
    {
        const TileCfg& c = s->buckets[(size_t)b].cfg;
        if (!tile_grid_ok(rq->out_w, rq->out_h, tile_w(s->threads, c), tile_h(s->threads, c)))
            return fail(CT_ERR_UNSUPPORTED, "request of %dx%d outputs spans more than %lld tiles along one side",
                        rq->out_w, rq->out_h, (long long)kMaxTilesPerSide);
    }
    auto r = std::make_shared<Request>();
    r->rq = *rq;
    r->bucket = b;
    std::unique_lock<std::mutex> g(s->mu);
    if (s->fatal != CT_OK) return fail((ct_status)s->fatal, "server stopped: %s", s->fatal_msg.c_str());
    if (rq->image_id) {
        auto it = s->images.find(rq->image_id);
        if (it == s->images.end()) return fail(CT_ERR_INVALID_ARG, "unknown image id");
        const Image& im = it->second;
        if (rq->out_w + rq->filter_w - 1 > im.in_w || rq->out_h + rq->filter_h - 1 > im.in_h)
            return fail(CT_ERR_INVALID_ARG, "request exceeds the resident image");
        r->own_image = false;
        r->d_image = s->base + im.off;
        r->in_pitch = im.in_pitch;
        it->second.users++;
    } else {
        if (!rq->h_image) return fail(CT_ERR_INVALID_ARG, "h_image or image_id is required");
        if (rq->in_pitch < rq->out_w + rq->filter_w - 1) return fail(CT_ERR_INVALID_ARG, "in_pitch < input width");
        const int64_t per16 = 16 / elem_size(s->o.dtype);
        r->in_pitch = round_up((int64_t)rq->out_w + rq->filter_w - 1, per16);   // compact device rows
        r->img_bytes = (size_t)(rq->out_h + rq->filter_h - 1) * (size_t)r->in_pitch * (size_t)elem_size(s->o.dtype);
    }
    r->out_dpitch = round_up(rq->out_w, 4);
    const size_t need = r->img_bytes + (size_t)rq->out_h * (size_t)r->out_dpitch * 4 + 1024;
    if (need > s->arena.size()) {
        if (!r->own_image) s->images[rq->image_id].users--;
        return fail(CT_ERR_OOM, "request needs %zu bytes, the budget is %zu", need, s->arena.size());
    }
    // filter taps, FP32, rows padded to 4
    const int fwp = (int)round_up(rq->filter_w, 4);
    r->taps.assign((size_t)rq->filter_h * fwp, 0.0f);
    for (int i = 0; i < rq->filter_h; ++i)
        for (int j = 0; j < rq->filter_w; ++j) {
            float v;
            const int k = i * rq->filter_w + j;
            if (s->o.dtype == CT_F32) {
                v = static_cast<const float*>(rq->h_filter)[k];
            } else {
                const uint32_t u = (uint32_t) static_cast<const uint16_t*>(rq->h_filter)[k] << 16;
                memcpy(&v, &u, 4);
            }
            r->taps[(size_t)i * fwp + j] = v;
        }
    int prev_dev = 0;
    cudaGetDevice(&prev_dev);
    if (prev_dev != s->device) cudaSetDevice(s->device);
    const cudaError_t ee = cudaEventCreateWithFlags(&r->ev_in, cudaEventDisableTiming);
    if (prev_dev != s->device) cudaSetDevice(prev_dev);
    if (ee != cudaSuccess) {
        if (!r->own_image) s->images[rq->image_id].users--;
        return fail(CT_ERR_CUDA, "cudaEventCreate");
    }
    r->id = s->next_id++;
    r->t_submit = now_s();
    if (s->submitted == 0 && s->completed == 0) s->t0 = r->t_submit;
    s->submitted++;
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    *request_id = r->id;
    g.unlock();
    s->cv_work.notify_one();
    return CT_OK;
}

CT_API ct_status ct_server_wait(ct_server* s, uint64_t request_id, int64_t timeout_us, double* latency_ms)
{
    if (!s) return fail(CT_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> g(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(CT_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)request_id);
    auto r = it->second;
    auto done = [&] { return r->state == RState::Done || r->state == RState::Failed; };
    if (timeout_us < 0) s->cv_done.wait(g, done);
    else if (!s->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), done))
        return fail(CT_ERR_TIMEOUT, "request %llu not done after %lld us", (unsigned long long)request_id,
                    (long long)timeout_us);
    if (latency_ms) *latency_ms = 1e3 * (r->t_done - r->t_submit);
    const int status = r->status;
    if (r->ev_in) cudaEventDestroy(r->ev_in);
    s->reqs.erase(it);
    if (status != CT_OK) return fail((ct_status)status, "request %llu failed", (unsigned long long)request_id);
    return CT_OK;
}

CT_API ct_status ct_server_drain(ct_server* s, int64_t timeout_us)
{
    if (!s) return fail(CT_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> g(s->mu);
    auto idle = [&] {
        bool busy = !s->pending.empty() || !s->admitted.empty() || !s->ready.empty();
        for (auto& L : s->launches) busy = busy || L.busy;
        return !busy;
    };
    if (timeout_us < 0) s->cv_done.wait(g, idle);
    else if (!s->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), idle))
        return fail(CT_ERR_TIMEOUT, "server not idle after %lld us", (long long)timeout_us);
    return CT_OK;
}

CT_API ct_status ct_server_stats_get(ct_server* s, ct_server_stats* out)
{
    if (!s || !out) return fail(CT_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->launches = s->n_launches;
    out->mean_batch = s->n_launches ? (double)s->launched_reqs / (double)s->n_launches : 0.0;
    out->peak_mem_bytes = (int64_t)s->arena.peak();
    std::vector<double> l = s->lat_ms;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
        auto q = [&](double p) {
            const size_t k = (size_t)std::ceil(p * (double)l.size());
            return l[std::min(l.size() - 1, k == 0 ? 0 : k - 1)];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = l.back();
        double m = 0;
        for (double x : l) m += x;
        out->mean_ms = m / (double)l.size();
    }
    out->wall_s = s->t_last - s->t0;
    if (out->wall_s > 0) {
        out->req_per_s = (double)s->completed / out->wall_s;
        out->gflops = s->flops / out->wall_s / 1e9;
    }
    // union of the kernel intervals
    std::vector<std::pair<float, float>> iv = s->kbusy;
    std::sort(iv.begin(), iv.end());
    double busy = 0.0, cur_a = 0.0, cur_b = -1.0;
    for (const auto& x : iv) {
        if (x.first > cur_b) {
            if (cur_b > cur_a) busy += cur_b - cur_a;
            cur_a = x.first;
            cur_b = x.second;
        } else {
            cur_b = std::max<double>(cur_b, x.second);
        }
    }
    if (cur_b > cur_a) busy += cur_b - cur_a;
    out->kernel_busy_s = busy * 1e-3;
    out->kernel_busy_frac = out->wall_s > 0 ? out->kernel_busy_s / out->wall_s : 0.0;
    return CT_OK;
}

CT_API ct_status ct_server_stats_reset(ct_server* s)
{
    if (!s) return fail(CT_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> g(s->mu);
    s->lat_ms.clear();
    s->kbusy.clear();
    s->submitted = s->completed = s->failed = s->n_launches = s->launched_reqs = 0;
    s->flops = 0;
    s->t0 = s->t_last = now_s();
    // new origin for the kernel intervals; launches still running keep the old one
    bool busy = false;
    for (auto& L : s->launches) busy = busy || L.busy;
    if (!busy) cudaEventRecord(s->ref, s->copy_in);
    return CT_OK;
}

CT_API ct_status ct_server_run(ct_server* s, const ct_server_run_opts* ro, ct_server_stats* out)
{
    if (!s || !ro || !ro->requests || ro->n <= 0 || ro->max_in_flight < 1)
        return fail(CT_ERR_INVALID_ARG, "server, options, requests (n > 0) and max_in_flight >= 1 are required");
    ct_status st = ct_server_drain(s, -1);
    if (st != CT_OK) return st;
    ct_server_stats_reset(s);
    const int64_t n = ro->n;
    std::vector<uint64_t> ids((size_t)n, 0);
    std::mutex m;
    std::condition_variable cv;
    int64_t n_sub = 0, n_done = 0;
    ct_status err = CT_OK, werr = CT_OK;
    std::string werr_msg;
    // completions are collected in submission order on a second thread
    std::thread waiter([&] {
        for (int64_t k = 0; k < n; ++k) {
            {
                std::unique_lock<std::mutex> g(m);
                cv.wait(g, [&] { return n_sub > k || err != CT_OK; });
                if (n_sub <= k) return;   // the submitter stopped
            }
            double lat = NAN;
            const ct_status w = ct_server_wait(s, ids[(size_t)k], ro->timeout_us, &lat);
            if (ro->latency_ms) ro->latency_ms[k] = w == CT_OK ? lat : NAN;
            std::lock_guard<std::mutex> g(m);
            if (w == CT_ERR_TIMEOUT && werr == CT_OK) {
                werr = w;
                werr_msg = last_error();
                err = w;
            }
            ++n_done;
            cv.notify_all();
            if (err != CT_OK && n_sub <= k + 1) return;
        }
    });
    const double t_start = now_s();
    for (int64_t k = 0; k < n; ++k) {
        if (ro->arrival_s) {
            const double due = t_start + ro->arrival_s[k];
            for (double now = now_s(); now < due; now = now_s())
                if (due - now > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        {
            std::unique_lock<std::mutex> g(m);
            cv.wait(g, [&] { return k - n_done < ro->max_in_flight || err != CT_OK; });
            if (err != CT_OK) break;
        }
        uint64_t id = 0;
        const ct_status sub = ct_server_submit(s, &ro->requests[k], &id);
        std::lock_guard<std::mutex> g(m);
        if (sub != CT_OK) {
            err = sub;
            werr_msg = last_error();
            cv.notify_all();
            break;
        }
        ids[(size_t)k] = id;
        n_sub = k + 1;
        cv.notify_all();
    }
    waiter.join();
    if (out) ct_server_stats_get(s, out);
    if (err != CT_OK) return fail(err, "server run stopped: %s", werr_msg.c_str());
    return CT_OK;
}

CT_API void ct_server_destroy(ct_server* s) { delete s; }

}  // extern "C"
