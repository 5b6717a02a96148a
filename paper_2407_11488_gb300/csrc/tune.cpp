// Runner and strategies: compile pool, event-timed benchmark of one variant,
// brute force / random sampling / simulated annealing, timing tables.
#include "ct_internal.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <limits>
#include <set>
#include <sstream>
#include <thread>

namespace ct {

// ---------------------------------------------------------- compile pool ---
CompilePool::CompilePool(int nthreads, std::string cache_dir, int reserve_urgent) : cache_dir_(std::move(cache_dir))
{
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
    max_speculative_ = (size_t)std::max(1, nthreads - std::max(0, reserve_urgent));
    for (int i = 0; i < nthreads; ++i) threads_.emplace_back([this] { worker(); });
}

CompilePool::~CompilePool()
{
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
        for (auto& q : queue_) q.pr->set_value(nullptr);
        queue_.clear();
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
}

std::shared_future<VariantPtr> CompilePool::request(const VariantKey& k, bool urgent)
{
    const std::string dir = cache_dir_;
    return request(k.packed(), [k, dir] { return compile_variant(k, dir); }, urgent);
}

std::shared_future<VariantPtr> CompilePool::request(uint64_t key, Job job, bool urgent)
{
    std::lock_guard<std::mutex> g(mu_);
    auto it = futures_.find(key);
    if (it != futures_.end()) {
        if (urgent) {
            for (auto q = queue_.begin(); q != queue_.end(); ++q)
                if (q->key == key) {
                    Item item = *q;
                    item.urgent = true;
                    queue_.erase(q);
                    queue_.push_front(item);
                    cv_.notify_all();
                    break;
                }
        }
        return it->second;
    }
    auto pr = std::make_shared<std::promise<VariantPtr>>();
    auto fut = pr->get_future().share();
    futures_[key] = fut;
    Item item{key, std::move(job), pr, urgent};
    if (urgent) queue_.push_front(std::move(item));
    else queue_.push_back(std::move(item));
    cv_.notify_all();
    return fut;
}

void CompilePool::forget(const VariantKey& k) { forget(k.packed()); }

bool CompilePool::ready(const VariantKey& k)
{
    std::lock_guard<std::mutex> g(mu_);
    auto it = futures_.find(k.packed());
    return it == futures_.end() || it->second.wait_for(std::chrono::seconds(0)) == std::future_status::ready;
}

size_t CompilePool::queued()
{
    std::lock_guard<std::mutex> g(mu_);
    return queue_.size();
}

void CompilePool::forget(uint64_t key)
{
    std::lock_guard<std::mutex> g(mu_);
    futures_.erase(key);
}

void CompilePool::worker()
{
    for (;;) {
        Item job;
        {
            std::unique_lock<std::mutex> g(mu_);
            cv_.wait(g, [this] {
                return stop_ ||
                       (!queue_.empty() && (queue_.front().urgent || running_speculative_ < max_speculative_));
            });
            if (stop_) return;
            job = queue_.front();
            queue_.pop_front();
            if (!job.urgent) ++running_speculative_;
        }
        job.pr->set_value(job.job());
        if (!job.urgent) {
            std::lock_guard<std::mutex> g(mu_);
            --running_speculative_;
            cv_.notify_all();
        }
    }
}

// ------------------------------------------------------------- measuring ---
struct Measure {
    int status = CT_OK;
    int n = 0;
    double med = NAN, mn = NAN, sd = NAN;   // of the faster grid
    double t_tiles = NAN, t_persist = NAN;  // medians per grid
    int persist = 0;                        // the faster grid
    int taps = 0;                           // 1: measured with the taps compiled in
    int fma2 = 0;                           // 1: measured with paired multiply-adds
    int sm_mhz = 0;
    int regs = 0, spill = 0;
    int64_t smem = 0;
    double compile_ms = 0.0;
};

static void summarize(std::vector<double>& t, Measure& m)
{
    std::sort(t.begin(), t.end());
    const size_t n = t.size();
    m.n = (int)n;
    if (!n) return;
    m.med = (n % 2) ? t[n / 2] : 0.5 * (t[n / 2 - 1] + t[n / 2]);
    m.mn = t[0];
    double mean = 0;
    for (double x : t) mean += x;
    mean /= (double)n;
    double ss = 0;
    for (double x : t) ss += (x - mean) * (x - mean);
    m.sd = n > 1 ? std::sqrt(ss / (double)(n - 1)) : 0.0;
}

class Evaluator {
public:
    virtual ~Evaluator() = default;
    virtual void prefetch(const Entry&, bool urgent = false) { (void)urgent; }
    virtual bool queue_short() const { return true; }
    // true when eval(e) would not wait for a compile
    virtual bool ready(const Entry&) { return true; }
    virtual Measure eval(const Entry& e) = 0;
    double compile_wait_ms = 0, compile_cpu_ms = 0, bench_ms = 0;
    bool abort = false;   // set after an unrecoverable device error
};

class ReplayEvaluator : public Evaluator {
public:
    ReplayEvaluator(const double* t, int64_t n) : t_(t), n_(n) {}
    Measure eval(const Entry& e) override
    {
        Measure m;
        const double v = e.index < n_ ? t_[e.index] : NAN;
        if (!(v > 0.0) || !std::isfinite(v)) {
            m.status = CT_ERR_LAUNCH;
            return m;
        }
        m.n = 1;
        m.med = m.mn = m.t_tiles = v;
        m.sd = 0.0;
        return m;
    }
private:
    const double* t_;
    int64_t n_;
};

struct TimeOpts {
    int repeats = 7, warmup = 1, flush_l2 = 0;
    double graph_below_ms = 0.05;
    int grid_modes = 0;   // 1: also time the persistent grid
    int taps_imm = 0;     // 1: unrolled variants get the problem's taps compiled in
    int sweep_fma2 = 0;   // 1: variants that admit it are measured with paired multiply-adds
};

class GpuEvaluator : public Evaluator {
public:
    GpuEvaluator(const ct_problem& p, const TimeOpts& o, const void* d_image, const void* h_filter, float* d_out,
                 CompilePool& pool, void* flush_buf, int64_t flush_bytes, cudaStream_t stream)
        : p_(p), o_(o), img_(d_image), filt_(h_filter), out_(d_out), pool_(pool), flush_(flush_buf),
          flush_bytes_(flush_bytes), s_(stream)
    {
        for (auto& e : ev_) cudaEventCreate(&e);
    }
    ~GpuEvaluator() override
    {
        for (auto& e : ev_) cudaEventDestroy(e);
    }
    VariantKey key(const Entry& e) const
    {
        ct_config c = e.cfg;
        c.taps = o_.taps_imm ? 1 : 0;
        c.fma2 = o_.sweep_fma2 ? 1 : 0;
        return variant_key(p_, c, filt_);
    }
    void prefetch(const Entry& e, bool urgent) override { pool_.request(key(e), urgent); }
    bool queue_short() const override { return pool_.queued() < 2 * pool_.threads(); }
    bool ready(const Entry& e) override { return pool_.ready(key(e)); }

    Measure eval(const Entry& e) override
    {
        Measure m;
        const VariantKey k = key(e);
        const double t0 = now_ms();
        VariantPtr v = pool_.request(k, true).get();   // needed now
        compile_wait_ms += now_ms() - t0;
        pool_.forget(k);
        if (!v) {
            m.status = CT_ERR_COMPILE;
            return m;
        }
        m.regs = v->regs;
        m.spill = v->spill_bytes;
        m.smem = v->smem;
        m.compile_ms = v->compile_ms;
        m.taps = k.taps.empty() ? 0 : 1;
        m.fma2 = k.cfg.fma2;
        compile_cpu_ms += v->compile_ms;
        if (v->status != CT_OK) {
            m.status = v->status;
            return m;
        }
        const double b0 = now_ms();
        m.status = time_variant(*v, m);
        bench_ms += now_ms() - b0;
        if (m.status == CT_OK && (!best_ || m.med < best_t_)) {
            best_ = v;
            best_t_ = m.med;
        } else {
            unload_variant(*v);
        }
        return m;
    }
    VariantPtr best() const { return best_; }
    ct_status fatal = CT_OK;

private:
    ct_status launch(Variant& v, int persist) { return launch_variant(v, p_, img_, filt_, out_, s_, persist); }

    // Times one grid form: warm-up launches, then the median of the timed ones.
    int time_variant(Variant& v, Measure& m)
    {
        ct_status s = load_variant(v);
        if (s != CT_OK) return s == CT_ERR_CUDA ? CT_ERR_LAUNCH : s;
        std::vector<double> t;
        int st = time_grid(v, 0, t);
        if (st != CT_OK) return st;
        summarize(t, m);
        m.t_tiles = m.med;
        m.persist = 0;
        if (o_.grid_modes && v.resident > 0 && tile_count(p_, v.key.cfg) > v.resident) {
            std::vector<double> t1;
            if ((st = time_grid(v, 1, t1)) != CT_OK) return st;
            Measure b;
            summarize(t1, b);
            m.t_persist = b.med;
            if (b.med < m.med) {
                m.n = b.n;
                m.med = b.med;
                m.mn = b.mn;
                m.sd = b.sd;
                m.persist = 1;
            }
        }
        if (take_device_error()) return CT_ERR_TIMEOUT;   // a launch gave up waiting for its input copy
        m.sm_mhz = sample_sm_mhz();
        return CT_OK;
    }

    int time_grid(Variant& v, int persist, std::vector<double>& t)
    {
        ct_status s;
        for (int w = 0; w < std::max(1, o_.warmup); ++w) {
            s = launch(v, persist);
            if (s != CT_OK) {
                cudaGetLastError();
                return CT_ERR_LAUNCH;
            }
        }
        cudaError_t e = cudaStreamSynchronize(s_);
        if (e != cudaSuccess) {
            fatal = cuda_fail(e, "kernel execution during tuning");
            abort = true;
            return CT_ERR_CUDA;
        }
        // one probe launch decides between single-launch and graph timing
        cudaEventRecord(ev_[0], s_);
        launch(v, persist);
        cudaEventRecord(ev_[1], s_);
        if ((e = cudaEventSynchronize(ev_[1])) != cudaSuccess) {
            fatal = cuda_fail(e, "kernel execution during tuning");
            abort = true;
            return CT_ERR_CUDA;
        }
        float probe = 0.f;
        cudaEventElapsedTime(&probe, ev_[0], ev_[1]);
        if (probe < o_.graph_below_ms) {
            const int K = std::min(1000, std::max(2, (int)std::ceil(0.5 / std::max(1e-4, (double)probe))));
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            if ((e = cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamBeginCapture"), CT_ERR_CUDA;
            bool ok = true;
            for (int i = 0; i < K && ok; ++i) ok = launch(v, persist) == CT_OK;
            e = cudaStreamEndCapture(s_, &g);
            if (!ok || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return CT_ERR_LAUNCH;
            }
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate"), CT_ERR_CUDA;
            cudaGraphLaunch(ge, s_);   // warm the graph
            for (int r = 0; r < o_.repeats; ++r) {
                cudaEventRecord(ev_[2 * (r % 16)], s_);
                cudaGraphLaunch(ge, s_);
                cudaEventRecord(ev_[2 * (r % 16) + 1], s_);
                if (r % 16 == 15 || r == o_.repeats - 1) {
                    cudaEventSynchronize(ev_[2 * (r % 16) + 1]);
                    for (int q = r - r % 16; q <= r; ++q) {
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, ev_[2 * (q % 16)], ev_[2 * (q % 16) + 1]);
                        t.push_back((double)ms / K);
                    }
                }
            }
            cudaGraphExecDestroy(ge);
        } else {
            for (int r = 0; r < o_.repeats; ++r) {
                if (o_.flush_l2 && flush_) launch_l2_flush(flush_, flush_bytes_, (uint32_t)r, s_);
                cudaEventRecord(ev_[2 * (r % 16)], s_);
                launch(v, persist);
                cudaEventRecord(ev_[2 * (r % 16) + 1], s_);
                if (r % 16 == 15 || r == o_.repeats - 1) {
                    cudaEventSynchronize(ev_[2 * (r % 16) + 1]);
                    for (int q = r - r % 16; q <= r; ++q) {
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, ev_[2 * (q % 16)], ev_[2 * (q % 16) + 1]);
                        t.push_back((double)ms);
                    }
                }
            }
        }
        if ((e = cudaStreamSynchronize(s_)) != cudaSuccess) {
            fatal = cuda_fail(e, "kernel execution during tuning");
            abort = true;
            return CT_ERR_CUDA;
        }
        return CT_OK;
    }

    ct_problem p_;
    TimeOpts o_;
    const void* img_;
    const void* filt_;
    float* out_;
    CompilePool& pool_;
    void* flush_;
    int64_t flush_bytes_;
    cudaStream_t s_;
    cudaEvent_t ev_[32];
    VariantPtr best_;
    double best_t_ = 0;
};

// ------------------------------------------------------------ table I/O ---
static std::string problem_tag(const ct_problem& p)
{
    char b[96];
    snprintf(b, sizeof b, "%dx%d/f%dx%d/%s", p.out_w, p.out_h, p.filter_w, p.filter_h,
             p.dtype == CT_BF16 ? "bf16" : "f32");
    return b;
}

static void fmt_num(std::ostringstream& os, double v)
{
    if (std::isfinite(v)) {
        char b[64];
        snprintf(b, sizeof b, "%.17g", v);
        os << b;
    } else {
        os << "null";
    }
}

static std::string row_json(const ct_row& r, const std::string& tag)
{
    std::ostringstream os;
    os << "{\"problem\":\"" << tag << "\",\"index\":" << r.index;
    for (int k = 0; k < 6; ++k) os << ",\"" << kParamNames[k] << "\":" << cfg_get(r.cfg, k);
    os << ",\"persist\":" << r.cfg.persist << ",\"taps\":" << r.cfg.taps << ",\"fma2\":" << r.cfg.fma2 << ",\"shfl\":" << r.cfg.shfl;
    os << ",\"status\":" << r.status << ",\"n\":" << r.n << ",\"t_med_ms\":";
    fmt_num(os, r.t_med_ms);
    os << ",\"t_min_ms\":";
    fmt_num(os, r.t_min_ms);
    os << ",\"t_std_ms\":";
    fmt_num(os, r.t_std_ms);
    os << ",\"gflops\":";
    fmt_num(os, r.gflops);
    os << ",\"regs\":" << r.regs << ",\"spill_bytes\":" << r.spill_bytes << ",\"smem_bytes\":" << r.smem_bytes
       << ",\"eval_order\":" << r.eval_order << ",\"compile_ms\":";
    fmt_num(os, r.compile_ms);
    os << ",\"t_tiles_ms\":";
    fmt_num(os, r.t_tiles_ms);
    os << ",\"t_persist_ms\":";
    fmt_num(os, r.t_persist_ms);
    os << ",\"t_remeasured_ms\":";
    fmt_num(os, r.t_remeasured_ms);
    os << ",\"sm_mhz\":" << r.sm_mhz << "}";
    return os.str();
}

static bool json_num(const std::string& line, const char* name, double& v)
{
    std::string pat = std::string("\"") + name + "\":";
    size_t pos = line.find(pat);
    if (pos == std::string::npos) return false;
    const char* s = line.c_str() + pos + pat.size();
    if (!strncmp(s, "null", 4)) {
        v = NAN;
        return true;
    }
    char* end = nullptr;
    v = strtod(s, &end);
    return end != s;
}

// Rows of an earlier run of the same problem, keyed by the packed config.
static std::unordered_map<uint64_t, Measure> read_resume(const char* path, const ct_problem& p)
{
    std::unordered_map<uint64_t, Measure> out;
    if (!path || !*path) return out;
    std::ifstream f(path);
    if (!f) return out;
    const std::string tag = "\"problem\":\"" + problem_tag(p) + "\"";
    std::string line;
    while (std::getline(f, line)) {
        if (line.find(tag) == std::string::npos) continue;
        ct_config c{};
        double v = 0;
        bool ok = true;
        for (int k = 0; k < 6; ++k) {
            ok = ok && json_num(line, kParamNames[k], v);
            cfg_set(c, k, (int)v);
        }
        Measure m;
        double st = 0, n = 0, r = 0, sp = 0, sm = 0, cm = 0;
        ok = ok && json_num(line, "status", st) && json_num(line, "n", n) && json_num(line, "t_med_ms", m.med) &&
             json_num(line, "t_min_ms", m.mn) && json_num(line, "t_std_ms", m.sd);
        if (!ok) continue;
        json_num(line, "regs", r);
        json_num(line, "spill_bytes", sp);
        json_num(line, "smem_bytes", sm);
        json_num(line, "compile_ms", cm);
        double pe = 0, tt = NAN, tp = NAN, mhz = 0, tk = 0;
        json_num(line, "persist", pe);
        json_num(line, "taps", tk);
        m.taps = tk == 1.0 ? 1 : 0;
        double f2 = 0;
        json_num(line, "fma2", f2);
        m.fma2 = f2 == 1.0 ? 1 : 0;
        if (!json_num(line, "t_tiles_ms", tt)) tt = m.med;
        json_num(line, "t_persist_ms", tp);
        json_num(line, "sm_mhz", mhz);
        m.persist = pe == 1.0 ? 1 : 0;
        m.t_tiles = tt;
        m.t_persist = tp;
        m.sm_mhz = (int)mhz;
        m.status = (int)st;
        m.n = (int)n;
        m.regs = (int)r;
        m.spill = (int)sp;
        m.smem = (int64_t)sm;
        m.compile_ms = std::isfinite(cm) ? cm : 0.0;
        out[VariantKey{c, p.filter_w, p.filter_h, p.dtype}.packed()] = m;
    }
    return out;
}

ct_status write_table(const ct_table& t, const char* path, const std::string& tag, bool append)
{
    FILE* f = fopen(path, append ? "a" : "w");
    if (!f) return fail(CT_ERR_INVALID_ARG, "cannot open %s for writing", path);
    for (const auto& r : t.rows) fprintf(f, "%s\n", row_json(r, tag).c_str());
    fclose(f);
    return CT_OK;
}

// ------------------------------------------------------------ strategies ---
class Driver {
public:
    Driver(const ct_problem& p, const Space& s, const std::vector<Entry>& valid, Evaluator& ev,
           std::unordered_map<uint64_t, Measure> resume, const char* append_path)
        : p_(p), s_(s), valid_(valid), ev_(ev), resume_(std::move(resume)), tag_(problem_tag(p))
    {
        for (size_t i = 0; i < valid_.size(); ++i) pos_[valid_[i].index] = i;
        if (append_path && *append_path) append_ = fopen(append_path, "a");
    }
    ~Driver()
    {
        if (append_) fclose(append_);
    }

    bool is_valid(int64_t idx) const { return pos_.count(idx) != 0; }
    bool queue_short() const { return ev_.queue_short(); }
    const Entry& entry(int64_t idx) const { return valid_[pos_.at(idx)]; }
    bool visited(int64_t idx) const { return row_of_.count(idx) != 0; }
    size_t n_rows() const { return rows.size(); }
    // true when evaluate(e) would not wait for a compile
    bool ready(const Entry& e)
    {
        return visited(e.index) || resume_.count(VariantKey{e.cfg, p_.filter_w, p_.filter_h, p_.dtype}.packed()) ||
               ev_.ready(e);
    }

    void prefetch(const Entry& e, bool urgent = false)
    {
        if (!visited(e.index) && !resume_.count(VariantKey{e.cfg, p_.filter_w, p_.filter_h, p_.dtype}.packed()))
            ev_.prefetch(e, urgent);
    }

    // Measures e once (memoised); returns its median time or +inf on failure.
    double evaluate(const Entry& e, bool* fresh = nullptr)
    {
        auto it = row_of_.find(e.index);
        if (fresh) *fresh = it == row_of_.end();
        if (it != row_of_.end()) return objective(rows[it->second]);
        Measure m;
        auto rit = resume_.find(VariantKey{e.cfg, p_.filter_w, p_.filter_h, p_.dtype}.packed());
        if (rit != resume_.end()) {
            m = rit->second;
        } else {
            m = ev_.eval(e);
        }
        ct_row r{};
        r.cfg = e.cfg;
        r.cfg.persist = m.status == CT_OK ? m.persist : 0;
        r.cfg.taps = m.taps;
        r.cfg.fma2 = m.fma2;
        r.t_tiles_ms = m.status == CT_OK ? m.t_tiles : NAN;
        r.t_persist_ms = m.status == CT_OK ? m.t_persist : NAN;
        r.t_remeasured_ms = NAN;
        r.sm_mhz = m.sm_mhz;
        r.index = e.index;
        r.status = m.status;
        r.n = m.n;
        r.t_med_ms = m.status == CT_OK ? m.med : NAN;
        r.t_min_ms = m.status == CT_OK ? m.mn : NAN;
        r.t_std_ms = m.status == CT_OK ? m.sd : NAN;
        r.gflops = m.status == CT_OK ? problem_flops(p_) / (m.med * 1e6) : 0.0;
        r.regs = m.regs;
        r.spill_bytes = m.spill;
        r.smem_bytes = (int32_t)m.smem;
        r.eval_order = (int32_t)rows.size();
        r.compile_ms = m.compile_ms;
        row_of_[e.index] = rows.size();
        rows.push_back(r);
        if (append_ && rit == resume_.end()) {
            fprintf(append_, "%s\n", row_json(r, tag_).c_str());
            fflush(append_);
        }
        return objective(r);
    }

    static double objective(const ct_row& r)
    {
        return r.status == CT_OK && std::isfinite(r.t_med_ms) ? r.t_med_ms : std::numeric_limits<double>::infinity();
    }

    std::vector<ct_row> rows;

private:
    const ct_problem& p_;
    const Space& s_;
    const std::vector<Entry>& valid_;
    Evaluator& ev_;
    std::unordered_map<uint64_t, Measure> resume_;
    std::string tag_;
    std::unordered_map<int64_t, size_t> pos_;
    std::unordered_map<int64_t, size_t> row_of_;
    FILE* append_ = nullptr;
};

static int64_t budget_of(const ct_tune_opts& o, int64_t n_valid)
{
    if (o.max_evals > 0) return std::min<int64_t>(o.max_evals, n_valid);
    const double f = o.sample_fraction > 0 ? o.sample_fraction : 0.10;
    return std::min<int64_t>(n_valid, std::max<int64_t>(1, (int64_t)std::ceil(f * (double)n_valid - 1e-9)));
}

static void run_list(Driver& d, const std::vector<Entry>& order, int window, const bool* stop)
{
    for (size_t i = 0; i < order.size(); ++i) {
        for (size_t j = i; j < std::min(order.size(), i + (size_t)window); ++j) d.prefetch(order[j]);
        d.evaluate(order[i]);
        if (stop && *stop) return;
    }
}

// Valid neighbours: one parameter moved by one step in its ordered value list.
static std::vector<int64_t> neighbours(const Space& s, const Driver& d, const ct_config& c)
{
    std::vector<int64_t> out;
    for (int k = 0; k < 6; ++k) {
        const auto& vals = s.vals[k];
        int pos = -1;
        for (size_t j = 0; j < vals.size(); ++j)
            if (vals[j] == cfg_get(c, k)) pos = (int)j;
        for (int dlt : {-1, 1}) {
            const int q = pos + dlt;
            if (pos < 0 || q < 0 || q >= (int)vals.size()) continue;
            ct_config n = c;
            cfg_set(n, k, vals[q]);
            const int64_t idx = s.index_of(n);
            if (idx >= 0 && d.is_valid(idx)) out.push_back(idx);
        }
    }
    return out;
}

// Simulated annealing over the valid configurations (neighbourhood as above),
// objective normalised by the first measured time, temperature cooled
// geometrically from 1 to 1e-3 over the evaluation budget, Metropolis
// acceptance, restart from the best point after budget/10 fresh evaluations
// without improvement, memoised measurements.  `chains` walkers each keep one
// candidate in flight (compiled as an urgent request, with the unmeasured
// neighbours of the walker's point and candidate compiled speculatively while
// the queue is short); the next candidate measured is that of the first
// walker, in round-robin order, whose compile has finished, so no walker
// waits for another's slow compile.  Without compiles (replay) every
// candidate is ready and the walkers take turns in order.  A restart moves
// every walker to the best point and replaces its candidate in flight by one
// proposed from there (a candidate proposed from the old point is dropped
// unmeasured).  `trace` (may be NULL) receives one JSON line per start point,
// step and restart.
static void run_anneal(Driver& d, const Space& s, const std::vector<Entry>& valid, int64_t budget, uint64_t seed,
                       int chains, const bool* stop, FILE* trace)
{
    Rng rng(seed ^ 0xA5A5A5A5ull);
    chains = std::max(1, std::min<int>(chains, (int)std::max<int64_t>(1, budget / 8)));
    struct Walker {
        const Entry* cur = nullptr;
        double f = std::numeric_limits<double>::infinity();
        int64_t idle = 0;
        const Entry* cand = nullptr;
        const Entry* from = nullptr;   // the point cand was proposed from
        bool jump = false;             // cand is a jump, not a neighbour of `from`
        int64_t epoch = 0;             // restarts before cand was proposed
    };
    int64_t epoch = 0;
    std::vector<Walker> w((size_t)chains);
    for (auto& x : w) x.cur = &valid[rng.below(valid.size())];
    for (auto& x : w) d.prefetch(*x.cur, true);
    double f_first = std::numeric_limits<double>::infinity();
    const Entry* best = w[0].cur;
    double f_best = std::numeric_limits<double>::infinity();
    for (size_t k = 0; k < w.size(); ++k) {
        Walker& x = w[k];
        x.f = d.evaluate(*x.cur);
        if (!std::isfinite(f_first) && std::isfinite(x.f)) f_first = x.f;
        if (x.f < f_best) { best = x.cur; f_best = x.f; }
        if (trace)
            fprintf(trace, "{\"ev\":\"start\",\"walker\":%zu,\"point\":%lld,\"f\":%.17g}\n", k,
                    (long long)x.cur->index, std::isfinite(x.f) ? x.f : -1.0);
    }
    // the next candidate of a walker: a random neighbour of its point, a
    // random unvisited point when it is stuck, or (on a failing point) a jump
    auto propose = [&](Walker& x) -> const Entry* {
        x.from = x.cur;
        x.jump = true;
        x.epoch = epoch;
        if (!std::isfinite(x.f)) {
            x.cur = &valid[rng.below(valid.size())];
            return x.cur;
        }
        std::vector<int64_t> nb = neighbours(s, d, x.cur->cfg);
        bool all_seen = true;
        for (int64_t i : nb) all_seen = all_seen && d.visited(i);
        if (nb.empty() || (all_seen && x.idle > 2 * (int64_t)nb.size())) {
            std::vector<const Entry*> fresh;
            for (const auto& e : valid)
                if (!d.visited(e.index)) fresh.push_back(&e);
            if (fresh.empty()) return nullptr;
            x.idle = 0;
            return fresh[rng.below(fresh.size())];
        }
        x.jump = false;
        return &d.entry(nb[rng.below(nb.size())]);
    };
    auto launch = [&](Walker& x) {
        x.cand = propose(x);
        if (!x.cand) return;
        d.prefetch(*x.cand, true);
        if (d.queue_short()) {   // speculative, behind the urgent requests
            for (int64_t i : neighbours(s, d, x.cur->cfg)) d.prefetch(d.entry(i), false);
            for (int64_t i : neighbours(s, d, x.cand->cfg)) d.prefetch(d.entry(i), false);
        }
    };
    for (auto& x : w) launch(x);
    const double T0 = 1.0, T1 = 1e-3;
    const int64_t stall_limit = std::max<int64_t>(1, budget / 10);
    int64_t stall = 0, steps = 0;
    const int64_t max_steps = 200 * budget + 1000;
    size_t rr = 0;
    while ((int64_t)d.n_rows() < budget && steps < max_steps) {
        if (stop && *stop) return;
        ++steps;
        // the first walker (round-robin) whose candidate is ready to measure
        size_t m = w.size();
        for (int spins = 0; m == w.size(); ++spins) {
            bool any = false;
            for (size_t k = 0; k < w.size(); ++k) {
                const size_t j = (rr + k) % w.size();
                if (!w[j].cand) continue;
                any = true;
                if (d.ready(*w[j].cand)) {
                    m = j;
                    break;
                }
            }
            if (!any) return;   // every point is visited
            if (m == w.size()) {
                if (spins > 200000) {   // ~20 s without a finished compile: measure the next in turn
                    for (size_t k = 0; k < w.size() && m == w.size(); ++k)
                        if (w[(rr + k) % w.size()].cand) m = (rr + k) % w.size();
                } else {
                    std::this_thread::sleep_for(std::chrono::microseconds(100));
                }
            }
        }
        rr = (m + 1) % w.size();
        Walker& x = w[m];
        bool fresh_eval = false;
        const double f_c = d.evaluate(*x.cand, &fresh_eval);
        if (!std::isfinite(f_first) && std::isfinite(f_c)) f_first = f_c;
        x.idle = fresh_eval ? 0 : x.idle + 1;
        bool accepted = false;
        if (!std::isfinite(x.f)) {
            x.cur = x.cand;
            x.f = f_c;
            accepted = true;
        } else if (std::isfinite(f_c)) {
            const double T = T0 * std::pow(T1 / T0, std::min(1.0, (double)d.n_rows() / (double)budget));
            const double delta = (f_c - x.f) / f_first;
            if (delta < 0 || rng.uniform() < std::exp(-delta / T)) {
                x.cur = x.cand;
                x.f = f_c;
                accepted = true;
            }
        }
        if (trace)
            fprintf(trace,
                    "{\"ev\":\"step\",\"walker\":%zu,\"epoch\":%lld,\"from\":%lld,\"cand\":%lld,\"jump\":%d,"
                    "\"fresh\":%d,\"accepted\":%d,\"f\":%.17g}\n",
                    m, (long long)x.epoch, (long long)(x.from ? x.from->index : -1), (long long)x.cand->index,
                    x.jump ? 1 : 0, fresh_eval ? 1 : 0, accepted ? 1 : 0, std::isfinite(f_c) ? f_c : -1.0);
        bool restart = false;
        if (f_c < f_best) {
            best = x.cand;
            f_best = f_c;
            stall = 0;
        } else if (fresh_eval && ++stall >= stall_limit) {
            restart = true;
            stall = 0;
        }
        if (restart) {
            ++epoch;
            if (trace)
                fprintf(trace, "{\"ev\":\"restart\",\"epoch\":%lld,\"best\":%lld,\"f\":%.17g}\n",
                        (long long)epoch, (long long)best->index, f_best);
            // every walker continues from the best point; candidates proposed
            // from the old points are replaced
            for (auto& y : w) {
                y.cur = best;
                y.f = f_best;
                y.idle = 0;
                if (&y != &x) launch(y);
            }
        }
        launch(x);
    }
}

static std::vector<Entry> random_sample(const std::vector<Entry>& valid, int64_t m, uint64_t seed)
{
    std::vector<size_t> idx(valid.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    Rng rng(seed);
    std::vector<Entry> out;
    for (int64_t i = 0; i < m; ++i) {
        const size_t j = (size_t)i + (size_t)rng.below(idx.size() - (size_t)i);
        std::swap(idx[(size_t)i], idx[j]);
        out.push_back(valid[idx[(size_t)i]]);
    }
    return out;
}

static ct_status run_strategy(const ct_problem& p, const Space& s, ct_strategy st, const ct_tune_opts& o,
                              const std::vector<Entry>& valid, Evaluator& ev, ct_table& t, int window)
{
    const bool* stop = &ev.abort;
    t.tag = problem_tag(p);
    Driver d(p, s, valid, ev, read_resume(o.resume_path, p), o.resume_path);
    const int64_t budget = budget_of(o, (int64_t)valid.size());
    if (st == CT_BRUTE) {
        run_list(d, valid, window, stop);
    } else if (st == CT_RANDOM) {
        run_list(d, random_sample(valid, budget, o.seed), window, stop);
    } else if (st == CT_ANNEAL) {
        FILE* trace = (o.trace_path && *o.trace_path) ? fopen(o.trace_path, "a") : nullptr;
        if (o.trace_path && *o.trace_path && !trace)
            return fail(CT_ERR_INVALID_ARG, "cannot open the trace file %s", o.trace_path);
        run_anneal(d, s, valid, budget, o.seed, o.anneal_chains > 0 ? o.anneal_chains : 1, stop, trace);
        if (trace) fclose(trace);
    } else {
        return fail(CT_ERR_INVALID_ARG, "unknown strategy %d", (int)st);
    }
    t.rows = std::move(d.rows);
    t.info.strategy = st;
    t.info.n_rows = (int32_t)t.rows.size();
    t.info.n_valid_space = (int64_t)valid.size();
    t.info.best_row = -1;
    for (size_t i = 0; i < t.rows.size(); ++i) {
        const ct_row& r = t.rows[i];
        if (r.status != CT_OK || !std::isfinite(r.t_med_ms)) continue;
        if (t.info.best_row < 0) {
            t.info.best_row = (int64_t)i;
            continue;
        }
        const ct_row& b = t.rows[(size_t)t.info.best_row];
        if (r.t_med_ms < b.t_med_ms || (r.t_med_ms == b.t_med_ms && r.index < b.index)) t.info.best_row = (int64_t)i;
    }
    t.info.compile_wall_ms = ev.compile_wait_ms;
    t.info.compile_cpu_ms = ev.compile_cpu_ms;
    t.info.bench_ms = ev.bench_ms;
    std::vector<int> mhz;
    for (const auto& r : t.rows)
        if (r.sm_mhz > 0) mhz.push_back(r.sm_mhz);
    if (!mhz.empty()) {
        std::nth_element(mhz.begin(), mhz.begin() + mhz.size() / 2, mhz.end());
        t.info.sm_mhz_median = mhz[mhz.size() / 2];
    }
    return CT_OK;
}

// Re-measures the k fastest rows (unless one of them ran for less than min_ms:
// short kernels keep their graph-timed figures) with `reps` launches each, interleaved
// round by round so that a clock change affects every candidate alike, each
// launch bracketed by events and preceded by the L2 flush when one is given.
// forms bit 0: an unrolled row is also timed in its other tap form (parameter
// block / compiled in); bit 1: also in the paired multiply-add form (two
// output rows per thread or more).  Each row keeps its fastest form
// (cfg.taps, cfg.fma2 record it).
// best_row becomes the fastest by the re-measured median.  Returns the
// variant of that row (null when nothing was re-measured).
static VariantPtr remeasure(ct_table& t, const ct_problem& p, int k, int reps, double min_ms, int forms,
                            const void* img, const void* filt, float* out, void* flush, int64_t flush_bytes,
                            cudaStream_t s, CompilePool& pool)
{
    std::vector<size_t> order;
    for (size_t i = 0; i < t.rows.size(); ++i) {
        const ct_row& r = t.rows[i];
        if (r.status == CT_OK && std::isfinite(r.t_med_ms)) order.push_back(i);
    }
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const ct_row &x = t.rows[a], &y = t.rows[b];
        return x.t_med_ms < y.t_med_ms || (x.t_med_ms == y.t_med_ms && x.index < y.index);
    });
    if ((int)order.size() > k) order.resize((size_t)k);
    // short kernels keep their graph-timed figures: when any of the fastest is
    // one, single launches would not compare with it, so nothing is re-measured
    for (size_t i : order)
        if (t.rows[i].t_med_ms < min_ms) return nullptr;
    if (order.size() < 2) return nullptr;
    const double t0 = now_ms();
    struct Cand {
        size_t row;
        ct_config cfg;
        VariantPtr v;
        std::vector<double> ms;
    };
    std::vector<Cand> cand;
    for (size_t i : order) {
        const ct_config c = t.rows[i].cfg;
        cand.push_back({i, c, nullptr, {}});
        if ((forms & 1) && c.unroll == 1) {
            ct_config alt = c;
            alt.taps = alt.taps ? 0 : 1;
            alt.fma2 = 0;
            const VariantKey vk = variant_key(p, alt, filt);
            if (vk.cfg.taps == alt.taps && vk.cfg.fma2 == 0) cand.push_back({i, alt, nullptr, {}});
        }
        if ((forms & 2) && c.unroll == 1 && !c.fma2) {
            ct_config alt = c;
            alt.taps = 0;
            alt.fma2 = 1;
            if (variant_key(p, alt, filt).cfg.fma2 == 1) cand.push_back({i, alt, nullptr, {}});
        }
        if ((forms & 4) && !c.shfl) {
            ct_config alt = c;
            alt.shfl = 1;
            if (variant_key(p, alt, filt).cfg.shfl == 1) cand.push_back({i, alt, nullptr, {}});
        }
    }
    std::vector<std::shared_future<VariantPtr>> futs;
    for (auto& c : cand) futs.push_back(pool.request(variant_key(p, c.cfg, filt), true));
    for (size_t j = 0; j < cand.size(); ++j) {
        cand[j].v = futs[j].get();
        pool.forget(variant_key(p, cand[j].cfg, filt));
        if (!cand[j].v || cand[j].v->status != CT_OK || load_variant(*cand[j].v) != CT_OK) return nullptr;
    }
    std::vector<cudaEvent_t> ev(2 * cand.size());
    for (auto& e : ev) cudaEventCreate(&e);
    bool ok = true;
    for (size_t j = 0; j < cand.size() && ok; ++j)   // warm-up
        ok = launch_variant(*cand[j].v, p, img, filt, out, s, cand[j].cfg.persist) == CT_OK;
    for (int r = 0; r < reps && ok; ++r) {
        for (size_t j = 0; j < cand.size() && ok; ++j) {
            if (flush) launch_l2_flush(flush, flush_bytes, (uint32_t)(r * 131 + j), s);
            cudaEventRecord(ev[2 * j], s);
            ok = launch_variant(*cand[j].v, p, img, filt, out, s, cand[j].cfg.persist) == CT_OK;
            cudaEventRecord(ev[2 * j + 1], s);
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
        for (size_t j = 0; j < cand.size() && ok; ++j) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * j], ev[2 * j + 1]);
            cand[j].ms.push_back((double)ms);
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (!ok || take_device_error()) {
        cudaGetLastError();
        return nullptr;
    }
    std::vector<VariantPtr> var_of(t.rows.size());
    for (auto& c : cand) {
        Measure m;
        summarize(c.ms, m);
        ct_row& row = t.rows[c.row];
        if (!std::isfinite(row.t_remeasured_ms) || m.med < row.t_remeasured_ms) {
            row.t_remeasured_ms = m.med;
            row.cfg.taps = c.cfg.taps;
            row.cfg.fma2 = c.cfg.fma2;
            row.cfg.shfl = c.cfg.shfl;
            var_of[c.row] = c.v;
        }
    }
    size_t best = order[0];
    for (size_t i : order) {
        const ct_row &x = t.rows[i], &b = t.rows[best];
        if (x.t_remeasured_ms < b.t_remeasured_ms || (x.t_remeasured_ms == b.t_remeasured_ms && x.index < b.index))
            best = i;
    }
    t.info.best_row = (int64_t)best;
    t.info.remeasured = (int32_t)order.size();
    t.info.remeasure_ms = now_ms() - t0;
    return var_of[best];
}

static ct_tune_opts normalise(const ct_tune_opts* o)
{
    ct_tune_opts r{};
    if (o) r = *o;
    if (r.repeats <= 0) r.repeats = 7;
    if (r.warmup <= 0) r.warmup = 1;
    if (r.graph_below_us == 0) r.graph_below_us = 50;
    if (r.remeasure_repeats <= 0) r.remeasure_repeats = 31;
    return r;
}

ct_status tune_replay(const ct_problem* p, const ct_space* s, ct_strategy st, const ct_tune_opts* opts,
                      const double* times, int64_t n_times, ct_config* best_out, ct_table** table_out)
{
    ct_status rc = check_problem(p);
    if (rc != CT_OK) return rc;
    if (!s || !times || !table_out) return fail(CT_ERR_INVALID_ARG, "space, times and table_out must be non-NULL");
    const double t0 = now_ms();
    ct_tune_opts o = normalise(opts);
    std::vector<Entry> valid = enumerate_valid(s->s, *p, kDefaultSmemLimit);
    if (valid.empty()) return fail(CT_ERR_INVALID_CONFIG, "no valid configuration in the space for this problem");
    ReplayEvaluator ev(times, n_times);
    auto* t = new ct_table();
    rc = run_strategy(*p, s->s, st, o, valid, ev, *t, 1);
    if (rc != CT_OK) {
        delete t;
        return rc;
    }
    t->info.wall_ms = now_ms() - t0;
    if (best_out && t->info.best_row >= 0) *best_out = t->rows[(size_t)t->info.best_row].cfg;
    *table_out = t;
    if (t->info.best_row < 0) return fail(CT_ERR_LAUNCH, "every evaluated configuration failed");
    return CT_OK;
}

ct_status tune_gpu(const ct_problem* p, const ct_space* s, ct_strategy st, const ct_tune_opts* opts,
                   const void* d_image, const void* h_filter, float* d_out, ct_config* best_out, ct_table** table_out)
{
    ct_status rc = check_problem(p);
    if (rc != CT_OK) return rc;
    if (!s || !table_out) return fail(CT_ERR_INVALID_ARG, "space and table_out must be non-NULL");
    if (p->out_w == 0 || p->out_h == 0) return fail(CT_ERR_INVALID_ARG, "cannot tune an empty problem");
    if ((rc = require_device()) != CT_OK) return rc;
    const double t0 = now_ms();
    ct_tune_opts o = normalise(opts);
    const int smem_limit = device_smem_limit();
    std::vector<Entry> valid = enumerate_valid(s->s, *p, smem_limit);
    if (valid.empty()) return fail(CT_ERR_INVALID_CONFIG, "no valid configuration in the space for this problem");

    cudaStream_t stream = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    void* img = nullptr;
    float* out = nullptr;
    void* flush = nullptr;
    int64_t flush_bytes = 0;
    std::vector<unsigned char> filt;
    auto cleanup = [&]() {
        cudaStreamSynchronize(stream);
        if (!d_image && img) cudaFree(img);
        if (!d_out && out) cudaFree(out);
        if (flush) cudaFree(flush);
        cudaStreamDestroy(stream);
    };
    const int es = elem_size(p->dtype);
    if (d_image) {
        img = const_cast<void*>(d_image);
    } else {
        if ((e = cudaMalloc(&img, (size_t)(in_h(*p) * p->in_pitch * es))) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "cudaMalloc(scratch image)");
        }
        cudaMemsetAsync(img, 0, (size_t)(in_h(*p) * p->in_pitch * es), stream);
        launch_fill_uniform(img, p->dtype, in_h(*p), in_w(*p), p->in_pitch, o.seed, 0, stream);
    }
    if (d_out) {
        out = d_out;
    } else if ((e = cudaMalloc((void**)&out, (size_t)(p->out_h * p->out_pitch * 4))) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMalloc(scratch output)");
    }
    if (!h_filter) {
        const int n = p->filter_w * p->filter_h;
        filt.resize((size_t)n * 4);
        const uint64_t start = (uint64_t)(in_w(*p) * in_h(*p));
        for (int i = 0; i < n; ++i) {
            const uint64_t u = splitmix64_at(o.seed, start + (uint64_t)i);
            const float v = (float)((double)(int64_t)(u >> 40) * 0x1p-23 - 1.0);
            if (p->dtype == CT_F32) {
                memcpy(&filt[(size_t)i * 4], &v, 4);
            } else {
                uint32_t b;
                memcpy(&b, &v, 4);
                b += 0x7fffu + ((b >> 16) & 1u);
                const uint16_t h = (uint16_t)(b >> 16);
                memcpy(&filt[(size_t)i * 2], &h, 2);
            }
        }
        h_filter = filt.data();
    }
    if (o.flush_l2) {
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        flush_bytes = 2 * (int64_t)std::max(l2, 64 << 20);
        if ((e = cudaMalloc(&flush, (size_t)flush_bytes)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "cudaMalloc(L2 flush buffer)");
        }
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "preparing tuning inputs");
    }
    TimeOpts to;
    to.repeats = o.repeats;
    to.warmup = o.warmup;
    to.flush_l2 = o.flush_l2;
    to.graph_below_ms = o.graph_below_us < 0 ? -1.0 : o.graph_below_us * 1e-3;
    to.grid_modes = o.grid_modes;
    to.taps_imm = o.taps_imm;
    to.sweep_fma2 = o.sweep_fma2;
    int threads = o.compile_threads > 0 ? o.compile_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    auto* t = new ct_table();
    {
        // annealing compiles its walkers' candidates urgently and their
        // neighbours speculatively: a quarter of the threads stay free for
        // the urgent ones, so a candidate never waits behind slow guesses
        CompilePool pool(threads, o.cache_dir ? std::string(o.cache_dir) : cache_dir_setting(),
                         st == CT_ANNEAL ? std::max(1, threads / 4) : 0);
        GpuEvaluator ev(*p, to, img, h_filter, out, pool, flush, flush_bytes, stream);
        rc = run_strategy(*p, s->s, st, o, valid, ev, *t, 2 * threads + 4);
        if (rc == CT_OK && ev.fatal != CT_OK) rc = ev.fatal;
        VariantPtr re;
        if (rc == CT_OK && o.remeasure_top > 0)
            re = remeasure(*t, *p, o.remeasure_top, o.remeasure_repeats, std::max(0.0, to.graph_below_ms),
                           o.remeasure_forms, img, h_filter, out, o.flush_l2 ? flush : nullptr, flush_bytes,
                           stream, pool);
        if (rc == CT_OK && re) put_variant(re);
        else if (rc == CT_OK && ev.best()) put_variant(ev.best());
    }
    cleanup();
    if (rc != CT_OK) {
        delete t;
        return rc;
    }
    t->info.wall_ms = now_ms() - t0;
    if (best_out && t->info.best_row >= 0) *best_out = t->rows[(size_t)t->info.best_row].cfg;
    *table_out = t;
    if (t->info.best_row < 0) return fail(CT_ERR_LAUNCH, "every evaluated configuration failed");
    return CT_OK;
}

}  // namespace ct
