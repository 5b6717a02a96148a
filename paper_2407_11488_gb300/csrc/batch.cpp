// Batched uneven correlations: bucketing, per-bucket tile tuning, work list,
// the persistent launch and its CUDA graph.
#include "batch_internal.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <numeric>

namespace ct {

static const char kBatchSource[] =
#include "batch_src.inc"
    ;

std::vector<std::string> batch_options(int threads, int dtype, const std::vector<BucketDesc>& b, int min_blocks)
{
    std::vector<std::string> o = nvrtc_base_options();
    auto def = [&](const std::string& n, int v) { o.push_back("-D" + n + "=" + std::to_string(v)); };
    def("CT_NT", threads);
    def("CT_DTYPE", dtype);
    def("CT_NB", (int)b.size());
    def("CT_MINB", min_blocks);
    int64_t buf = 128;
    for (const auto& d : b) buf = std::max(buf, bucket_buf_bytes(threads, d.cfg, d.fw, d.fh, dtype));
    def("CT_BUF_BYTES", (int)buf);
    for (size_t k = 0; k < b.size(); ++k) {
        const std::string p = "CT_B" + std::to_string(k) + "_";
        def(p + "BX", b[k].cfg.bx);
        def(p + "TX", b[k].cfg.tx);
        def(p + "TY", b[k].cfg.ty);
        def(p + "FW", b[k].fw);
        def(p + "FH", b[k].fh);
        def(p + "UN", b[k].cfg.un);
        def(p + "P2", b[k].cfg.p2);
    }
    add_env_options(o);
    return o;
}

uint64_t options_key(const std::vector<std::string>& o)
{
    uint64_t h = 1469598103934665603ull ^ 0xB47C4ull;
    for (const auto& s : o)
        for (size_t i = 0; i <= s.size(); ++i) {
            h ^= (unsigned char)(i < s.size() ? s[i] : 0);
            h *= 1099511628211ull;
        }
    return h;
}

VariantPtr compile_batch(int threads, int dtype, const std::vector<BucketDesc>& b, const std::string& dir,
                         int min_blocks)
{
    VariantPtr v = compile_source(kBatchSource, sizeof kBatchSource, "batch.cu",
                                  batch_options(threads, dtype, b, min_blocks), "ct_corr2d_batch", dir);
    int64_t sm = 0;
    for (const auto& d : b) sm = std::max(sm, bucket_smem(threads, d.cfg, d.fw, d.fh, dtype));
    v->smem = sm;
    return v;
}


ct_status launch_batch(Variant& v, int grid, int threads, const DevParams& prm, cudaStream_t s)
{
    ct_status st = load_variant(v);
    if (st != CT_OK) return st;
    DevParams copy = prm;
    void* args[1] = {&copy};
    cudaError_t e = cudaLaunchKernel((const void*)v.kern, dim3((unsigned)grid), dim3((unsigned)threads), args,
                                     (size_t)v.smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernel(ct_corr2d_batch)");
    return CT_OK;
}

int occupancy_grid(Variant& v, int threads, int blocks_per_sm, int64_t n_work)
{
    int dev = 0, sms = 1, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks_per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)v.kern, threads, (size_t)v.smem) !=
                cudaSuccess ||
            nb <= 0) {
            cudaGetLastError();
            nb = 1;
        }
    } else {
        nb = blocks_per_sm;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb * sms, n_work));
}

}  // namespace ct

using namespace ct;

struct ct_batch {
    struct Bucket {
        int fw = 0, fh = 0, side = 0;
        std::vector<int> items;
        TileCfg cfg;
        double pp = NAN;
    };
    int dtype = CT_F32, threads = 256, min_blocks = kMinBlocks;
    std::vector<ct_batch_item> items;
    std::vector<int> item_bucket;
    std::vector<int> filt_off;
    std::vector<Bucket> buckets;
    VariantPtr module;
    // problems run as their own single-problem launch, with their variant
    std::vector<int> solo_items;
    std::vector<VariantPtr> solo_vars;
    void* d_probs = nullptr;
    void* d_work = nullptr;
    float* d_filters = nullptr;
    void* d_tmaps = nullptr;
    unsigned* d_counter = nullptr;
    int64_t n_work = 0;
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    ct_batch_info info{};
    ~ct_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (d_probs) cudaFree(d_probs);
        if (d_work) cudaFree(d_work);
        if (d_filters) cudaFree(d_filters);
        if (d_tmaps) cudaFree(d_tmaps);
        if (d_counter) cudaFree(d_counter);
    }
};

namespace {

int64_t tiles_of(const ct_batch_item& it, int threads, const TileCfg& c, int64_t* tx_out = nullptr)
{
    if (it.out_w <= 0 || it.out_h <= 0) {
        if (tx_out) *tx_out = 0;
        return 0;
    }
    const int64_t tw = tile_w(threads, c), th = tile_h(threads, c);
    const int64_t tx = (it.out_w + tw - 1) / tw, ty = (it.out_h + th - 1) / th;
    if (tx_out) *tx_out = tx;
    return tx * ty;
}

DevProblem dev_problem(const ct_batch& B, int i, int bucket, const TileCfg& c)
{
    const ct_batch_item& it = B.items[(size_t)i];
    DevProblem d{};
    d.in = it.d_image;
    d.out = it.d_out;
    d.in_pitch = it.in_pitch;
    d.out_pitch = it.out_pitch;
    d.out_w = it.out_w;
    d.out_h = it.out_h;
    d.in_w = it.out_w + it.filter_w - 1;
    d.in_h = it.out_h + it.filter_h - 1;
    d.bucket = bucket;
    int64_t tx = 0;
    tiles_of(it, B.threads, c, &tx);
    d.tiles_x = (int32_t)tx;
    d.filt_off = B.filt_off[(size_t)i];
    return d;
}

// Tensor map of item i's image for the halo box of tile configuration c
// (all zero for an empty item, which has no tiles).
ct_status item_map(const ct_batch& B, int i, const TileCfg& c, unsigned char* map)
{
    const ct_batch_item& it = B.items[(size_t)i];
    memset(map, 0, kTensorMapBytes);
    if (it.out_w == 0 || it.out_h == 0) return CT_OK;
    return encode_halo_map(map, it.d_image, B.dtype, it.out_w + it.filter_w - 1, it.out_h + it.filter_h - 1,
                           it.in_pitch, batch_box_w(B.threads, c, it.filter_w, B.dtype),
                           batch_box_h(B.threads, c, it.filter_h));
}

// Candidate tiles of one bucket: block width, register tile, row-loop
// unrolling; the halo box must suit a tensor copy, the two item buffers must
// leave room for min_blocks blocks per SM, and a fully unrolled body stays
// below ~6k FMAs (instruction cache).
// forms: 0 scalar and paired multiply-adds, 1 scalar only, 2 paired only
// (scalar where no paired tile fits).
std::vector<TileCfg> bucket_candidates(int threads, int fw, int fh, int dtype, int smem_limit, int min_blocks,
                                       int forms)
{
    std::vector<TileCfg> out;
    const int64_t cap = std::min<int64_t>(smem_limit, (int64_t)kSmemPerSM / std::max(1, min_blocks) - 1024);
    for (int bx : {16, 32, 64}) {
        if (bx > threads || threads % bx) continue;
        for (int tx : {2, 4, 8})
            for (int ty : {1, 2, 4, 8})
                for (int un : {0, 1})
                    for (int p2 : {0, 1}) {
                        TileCfg c{bx, tx, ty, un, p2};
                        if (p2 && (forms == 1 || !pair_ok(c))) continue;
                        if (!halo_box_ok(threads, c, fw, fh, dtype)) continue;
                        if (bucket_smem(threads, c, fw, fh, dtype) > cap) continue;
                        if (un && (int64_t)tx * ty * fw * (fh + ty - 1) > 6144) continue;
                        out.push_back(c);
                    }
    }
    if (forms == 2 && std::any_of(out.begin(), out.end(), [](const TileCfg& c) { return c.p2 != 0; }))
        out.erase(std::remove_if(out.begin(), out.end(), [](const TileCfg& c) { return c.p2 == 0; }), out.end());
    return out;
}

// Measures every candidate tile on (a sample of) the bucket's problems and
// picks the one with the best objective.
ct_status tune_bucket(ct_batch& B, ct_batch::Bucket& bk, const ct_batch_opts& o, CompilePool& pool,
                      cudaStream_t s, int smem_limit)
{
    std::vector<TileCfg> cand =
        bucket_candidates(B.threads, bk.fw, bk.fh, B.dtype, smem_limit, B.min_blocks, o.bucket_forms);
    if (cand.empty())
        return fail(CT_ERR_INVALID_CONFIG, "no tile fits shared memory and the tensor copy for filter %dx%d", bk.fw,
                    bk.fh);
    // sample of problems: sorted by size, evenly spaced, always the extremes
    std::vector<int> its = bk.items;
    std::sort(its.begin(), its.end(), [&](int a, int b) {
        return (int64_t)B.items[(size_t)a].out_w * B.items[(size_t)a].out_h >
               (int64_t)B.items[(size_t)b].out_w * B.items[(size_t)b].out_h;
    });
    its.erase(std::remove_if(its.begin(), its.end(),
                             [&](int i) { return B.items[(size_t)i].out_w == 0 || B.items[(size_t)i].out_h == 0; }),
              its.end());
    if (its.empty()) return CT_OK;
    const size_t cap = (size_t)(o.max_tune_items > 0 ? o.max_tune_items : 12);
    std::vector<int> sample;
    if (its.size() <= cap) {
        sample = its;
    } else {
        for (size_t k = 0; k < cap; ++k) sample.push_back(its[k * (its.size() - 1) / (cap - 1)]);
        sample.erase(std::unique(sample.begin(), sample.end()), sample.end());
    }
    cand.erase(std::remove_if(cand.begin(), cand.end(),
                              [&](const TileCfg& c) {
                                  for (int i : sample)
                                      if (!tile_grid_ok(B.items[(size_t)i].out_w, B.items[(size_t)i].out_h,
                                                        tile_w(B.threads, c), tile_h(B.threads, c)))
                                          return true;
                                  return false;
                              }),
               cand.end());
    if (cand.empty()) return fail(CT_ERR_UNSUPPORTED, "no tile keeps the bucket's problems within %lld tiles a side",
                                  (long long)kMaxTilesPerSide);
    // compile all candidates in parallel
    std::vector<std::shared_future<VariantPtr>> futs;
    std::vector<uint64_t> keys;
    for (const auto& c : cand) {
        std::vector<BucketDesc> one = {{bk.fw, bk.fh, c}};
        const uint64_t key = options_key(batch_options(B.threads, B.dtype, one, B.min_blocks));
        const std::string dir = pool.cache_dir();
        const int thr = B.threads, dt = B.dtype, mb = B.min_blocks;
        keys.push_back(key);
        futs.push_back(pool.request(key, [thr, dt, one, dir, mb] { return compile_batch(thr, dt, one, dir, mb); }));
    }
    int64_t max_tiles = 1;
    for (const auto& c : cand)
        for (int i : sample) max_tiles = std::max(max_tiles, tiles_of(B.items[(size_t)i], B.threads, c));
    void* d_prob = nullptr;
    void* d_work = nullptr;
    void* d_map = nullptr;
    unsigned* d_cnt = nullptr;
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        if (d_prob) cudaFree(d_prob);
        if (d_work) cudaFree(d_work);
        if (d_map) cudaFree(d_map);
        if (d_cnt) cudaFree(d_cnt);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        for (auto k : keys) pool.forget(k);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&d_prob, sizeof(DevProblem))) != cudaSuccess ||
        (e = cudaMalloc(&d_work, (size_t)max_tiles * sizeof(WorkItem))) != cudaSuccess ||
        (e = cudaMalloc(&d_map, kTensorMapBytes)) != cudaSuccess ||
        (e = cudaMalloc((void**)&d_cnt, kCounterWords * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemsetAsync(d_cnt, 0, kCounterWords * sizeof(unsigned), s)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMalloc(batch tuning scratch)");
    }
    alignas(64) unsigned char map[kTensorMapBytes];
    const size_t nc = cand.size(), ni = sample.size();
    std::vector<double> t((size_t)(nc * ni), std::numeric_limits<double>::infinity());
    std::vector<WorkItem> work;
    for (size_t ci = 0; ci < nc; ++ci) {
        VariantPtr v = futs[ci].get();
        if (!v || v->status != CT_OK) continue;
        for (size_t ii = 0; ii < ni; ++ii) {
            const int item = sample[ii];
            const DevProblem dp = dev_problem(B, item, 0, cand[ci]);
            ct_status st = item_map(B, item, cand[ci], map);
            if (st != CT_OK) {
                cleanup();
                return st;
            }
            int64_t tx = 0;
            const int64_t nt = tiles_of(B.items[(size_t)item], B.threads, cand[ci], &tx);
            work.resize((size_t)nt);
            for (int64_t k = 0; k < nt; ++k) work[(size_t)k] = work_item(0u, k, tx, 0, dp.filt_off);
            cudaMemcpyAsync(d_prob, &dp, sizeof dp, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(d_work, work.data(), (size_t)nt * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(d_map, map, kTensorMapBytes, cudaMemcpyHostToDevice, s);
            if ((st = load_variant(*v)) != CT_OK) break;
            const int grid = occupancy_grid(*v, B.threads, o.blocks_per_sm, nt);
            DevParams prm{d_prob, d_work, B.d_filters, d_map, d_cnt, (int32_t)nt, 0};
            std::vector<float> ms;
            bool ok = true;
            for (int r = 0; r < 4 && ok; ++r) {
                cudaMemsetAsync(d_cnt, 0, sizeof(unsigned), s);
                cudaEventRecord(ev[0], s);
                ok = launch_batch(*v, grid, B.threads, prm, s) == CT_OK;
                cudaEventRecord(ev[1], s);
                if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) {
                    cleanup();
                    return cuda_fail(e, "batch tuning launch");
                }
                float x = 0.f;
                cudaEventElapsedTime(&x, ev[0], ev[1]);
                if (r > 0) ms.push_back(x);   // the first launch is a warm-up
            }
            if (!ok) {
                cudaGetLastError();
                continue;
            }
            std::sort(ms.begin(), ms.end());
            t[ci * ni + ii] = ms[ms.size() / 2];
        }
        unload_variant(*v);
    }
    cleanup();
    // objective
    size_t best = nc;
    double best_score = -1.0;
    double best_pp = NAN;
    std::vector<double> pmax(ni, 0.0);
    for (size_t ii = 0; ii < ni; ++ii)
        for (size_t ci = 0; ci < nc; ++ci)
            if (std::isfinite(t[ci * ni + ii])) pmax[ii] = std::max(pmax[ii], 1.0 / t[ci * ni + ii]);
    for (size_t ci = 0; ci < nc; ++ci) {
        double inv = 0.0, sum_t = 0.0;
        bool all = true;
        for (size_t ii = 0; ii < ni; ++ii) {
            const double x = t[ci * ni + ii];
            if (!std::isfinite(x)) {
                all = false;
                break;
            }
            inv += pmax[ii] * x;   // 1 / e_i with e_i = (1/x) / pmax_i
            sum_t += x;
        }
        if (!all) continue;
        const double pp = (double)ni / inv;
        const double score = o.objective == 1 ? 1.0 / sum_t : pp;
        if (score > best_score) {
            best_score = score;
            best = ci;
            best_pp = pp;
        }
    }
    if (best == nc) return fail(CT_ERR_LAUNCH, "no tile configuration ran for filter %dx%d", bk.fw, bk.fh);
    bk.cfg = cand[best];
    bk.pp = best_pp;
    return CT_OK;
}

// Problems that fill at least `pct` percent of one wave of the GPU on their
// own go solo.  For every filter size whose largest problem could (one output
// per resident thread), the single-problem configuration is tuned on that
// problem (annealing, o.solo_evals evaluations, on its own buffers); each
// problem of that size whose tile count under the configuration reaches
// pct/100 x SMs x resident blocks then runs as its own launch of it.
ct_status plan_solo(ct_batch& B, const ct_batch_opts& o, std::vector<char>& solo, double* tune_ms)
{
    const int pct = o.solo_wave_pct == 0 ? 10 : o.solo_wave_pct;
    if (pct <= 0) return CT_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int n = (int)B.items.size();
    auto area = [&](int i) { return (int64_t)B.items[(size_t)i].out_w * B.items[(size_t)i].out_h; };
    std::map<std::pair<int, int>, int> largest;
    for (int i = 0; i < n; ++i) {
        if (area(i) * 100 < (int64_t)pct * sms * 2048) continue;
        const auto key = std::make_pair(B.items[(size_t)i].filter_w, B.items[(size_t)i].filter_h);
        auto f = largest.find(key);
        if (f == largest.end() || area(i) > area(f->second)) largest[key] = i;
    }
    if (largest.empty()) return CT_OK;
    const double t0 = now_ms();
    ct_space* sp = nullptr;
    ct_status st = ct_space_builtin("full", &sp);
    if (st != CT_OK) return st;
    struct SpaceGuard {
        ct_space* s;
        ~SpaceGuard() { ct_space_free(s); }
    } sg{sp};
    std::vector<std::pair<int64_t, int>> picked;   // (area, item)
    std::map<int, VariantPtr> var_of;
    for (const auto& kv : largest) {
        const ct_batch_item& big = B.items[(size_t)kv.second];
        const ct_problem p{big.out_w, big.out_h, big.filter_w, big.filter_h, big.in_pitch, big.out_pitch, B.dtype, 0};
        ct_tune_opts to{};
        to.seed = 1;
        to.max_evals = o.solo_evals > 0 ? o.solo_evals : 60;
        to.anneal_chains = 4;
        // the five fastest are timed again, also with paired multiply-adds (a
        // form every problem of the size can share: taps stay in the parameter block)
        to.remeasure_top = 5;
        to.remeasure_forms = 2;
        ct_config best{};
        ct_table* t = nullptr;
        st = ct_tune(&p, sp, CT_ANNEAL, &to, big.d_image, big.h_filter, big.d_out, &best, &t);
        if (t) ct_table_free(t);
        if (st == CT_ERR_CUDA)
            return fail(st, "tuning the single-problem configuration for filter %dx%d: %s", big.filter_w,
                        big.filter_h, last_error());
        if (st != CT_OK) continue;   // no configuration ran: this size stays in the persistent launch
        // one variant per filter size, shared by problems with different filters: taps in the parameter block
        best.taps = 0;
        VariantPtr v = compile_variant(variant_key(p, best, nullptr), cache_dir_setting());
        if (!v || v->status != CT_OK)
            return fail(CT_ERR_COMPILE, "single-problem variant: %s", v ? v->error.c_str() : "no variant");
        if ((st = load_variant(*v)) != CT_OK) return st;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)v->kern, best.block_x * best.block_y,
                                                          (size_t)v->smem) != cudaSuccess ||
            nb <= 0) {
            cudaGetLastError();
            nb = 1;
        }
        const int64_t slots = std::max<int64_t>(1, (int64_t)pct * sms * nb / 100);
        const int64_t tw = (int64_t)best.block_x * best.tile_x, th = (int64_t)best.block_y * best.tile_y;
        for (int i = 0; i < n; ++i) {
            const ct_batch_item& it = B.items[(size_t)i];
            if (it.filter_w != big.filter_w || it.filter_h != big.filter_h) continue;
            if (((it.out_w + tw - 1) / tw) * ((it.out_h + th - 1) / th) < slots) continue;
            solo[(size_t)i] = 1;
            picked.emplace_back(area(i), i);
            var_of[i] = v;
        }
    }
    std::stable_sort(picked.begin(), picked.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (const auto& pi : picked) {
        B.solo_items.push_back(pi.second);
        B.solo_vars.push_back(var_of[pi.second]);
    }
    *tune_ms = now_ms() - t0;
    return CT_OK;
}

}  // namespace

extern "C" {

CT_API ct_status ct_batch_create(const ct_batch_item* items, int32_t n, const ct_batch_opts* opts, ct_batch** out)
{
    if (!out) return fail(CT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !items) return fail(CT_ERR_INVALID_ARG, "a batch needs at least one item");
    ct_batch_opts o{};
    if (opts) o = *opts;
    if (o.dtype != CT_F32 && o.dtype != CT_BF16) return fail(CT_ERR_INVALID_ARG, "bad batch dtype %d", o.dtype);
    const int threads = o.threads > 0 ? o.threads : 256;
    if (threads % 16 || threads > 1024) return fail(CT_ERR_INVALID_ARG, "threads must be a multiple of 16, <= 1024");
    if (o.min_blocks_per_sm < 0 || o.min_blocks_per_sm > 8)
        return fail(CT_ERR_INVALID_ARG, "min_blocks_per_sm must be 0..8");
    const int split = o.side_split == 0 ? 512 : o.side_split;
    ct_status st;
    for (int i = 0; i < n; ++i) {
        const ct_batch_item& it = items[i];
        ct_problem p{it.out_w, it.out_h, it.filter_w, it.filter_h, it.in_pitch, it.out_pitch, o.dtype, 0};
        if ((st = check_problem(&p)) != CT_OK || (st = check_buffers(p, it.d_image, it.h_filter, it.d_out)) != CT_OK)
            return fail(st, "batch item %d: %s", i, last_error());
    }
    if ((st = require_device()) != CT_OK) return st;
    const double t0 = now_ms();
    auto B = std::unique_ptr<ct_batch>(new ct_batch());
    B->dtype = o.dtype;
    B->threads = threads;
    B->min_blocks = o.min_blocks_per_sm > 0 ? o.min_blocks_per_sm : kMinBlocks;
    B->items.assign(items, items + n);
    // filters, widened to FP32, in one arena: per filter its zero-padded tap
    // rows and its rows of tap pairs (every filter starts on a 16-byte boundary)
    std::vector<float> arena, f32;
    for (int i = 0; i < n; ++i) {
        const ct_batch_item& it = items[i];
        const int nf = it.filter_w * it.filter_h;
        f32.resize((size_t)nf);
        for (int k = 0; k < nf; ++k) {
            if (o.dtype == CT_F32) {
                f32[(size_t)k] = static_cast<const float*>(it.h_filter)[k];
            } else {
                const uint32_t u = (uint32_t) static_cast<const uint16_t*>(it.h_filter)[k] << 16;
                memcpy(&f32[(size_t)k], &u, 4);
            }
        }
        const int64_t off = append_filter(arena, f32.data(), it.filter_w, it.filter_h);
        if (off > (int64_t)0x7fffffff) return fail(CT_ERR_UNSUPPORTED, "filter table too large");
        B->filt_off.push_back((int)off);
    }
    // problems that fill the GPU alone run as their own launch of the
    // single-problem kernel (constant-bank taps), configuration tuned per
    // filter size on its largest problem
    B->item_bucket.assign((size_t)n, -1);
    std::vector<char> solo((size_t)n, 0);
    double solo_tune_ms = 0.0;
    if ((st = plan_solo(*B, o, solo, &solo_tune_ms)) != CT_OK) return st;
    // buckets: filter size, then image side class
    for (int pass = 0; pass < 2; ++pass) {
        B->buckets.clear();
        for (int i = 0; i < n; ++i) {
            const ct_batch_item& it = items[i];
            if (solo[(size_t)i]) continue;
            const int side = (pass == 0 && split > 0 && std::max(it.out_w, it.out_h) >= split) ? 1 : 0;
            int k = -1;
            for (size_t b = 0; b < B->buckets.size(); ++b)
                if (B->buckets[b].fw == it.filter_w && B->buckets[b].fh == it.filter_h && B->buckets[b].side == side)
                    k = (int)b;
            if (k < 0) {
                ct_batch::Bucket nb;
                nb.fw = it.filter_w;
                nb.fh = it.filter_h;
                nb.side = side;
                B->buckets.push_back(nb);
                k = (int)B->buckets.size() - 1;
            }
            B->buckets[(size_t)k].items.push_back(i);
            B->item_bucket[(size_t)i] = k;
        }
        if (B->buckets.size() <= 16) break;
    }
    if (B->buckets.size() > 16) return fail(CT_ERR_UNSUPPORTED, "more than 16 filter sizes in one batch");
    cudaError_t e;
    if ((e = cudaMalloc((void**)&B->d_filters, std::max<size_t>(4, arena.size() * 4))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(batch filters)");
    if ((e = cudaMemcpy(B->d_filters, arena.data(), arena.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload batch filters");
    const int smem_limit = device_smem_limit();
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } sg{s};
    double compile_cpu = 0.0;
    const double tt0 = now_ms();
    {
        CompilePool pool(0, cache_dir_setting());
        for (auto& bk : B->buckets) {
            if (o.tune) {
                if ((st = tune_bucket(*B, bk, o, pool, s, smem_limit)) != CT_OK) return st;
            } else {
                // fixed default tile; bucket_forms = 2 asks for its paired form
                bk.cfg = o.bucket_forms == 2 ? TileCfg{32, 4, 4, 1, 1} : TileCfg{32, 4, 4, 0, 0};
                if (threads % 32) bk.cfg.bx = 16;
                while ((bucket_smem(threads, bk.cfg, bk.fw, bk.fh, o.dtype) > smem_limit ||
                        !halo_box_ok(threads, bk.cfg, bk.fw, bk.fh, o.dtype)) &&
                       bk.cfg.ty > 1)
                    bk.cfg.ty /= 2;
                if (bk.cfg.p2 && (!pair_ok(bk.cfg) ||
                                  (int64_t)bk.cfg.tx * bk.cfg.ty * bk.fw * (bk.fh + bk.cfg.ty - 1) > 6144))
                    bk.cfg = TileCfg{bk.cfg.bx, bk.cfg.tx, bk.cfg.ty, 0, 0};
                if (!halo_box_ok(threads, bk.cfg, bk.fw, bk.fh, o.dtype))
                    return fail(CT_ERR_UNSUPPORTED, "no default tile suits a tensor copy with %d threads", threads);
            }
        }
    }
    B->info.tune_ms = (o.tune ? now_ms() - tt0 : 0.0) + solo_tune_ms;
    const bool persistent = !B->buckets.empty();
    std::vector<DevProblem> probs;
    std::vector<unsigned char> maps((size_t)n * kTensorMapBytes, 0);
    std::vector<WorkItem> work;
    if (persistent) {
        // the persistent kernel with every bucket's tile routine
        std::vector<BucketDesc> desc;
        for (const auto& bk : B->buckets) desc.push_back({bk.fw, bk.fh, bk.cfg});
        B->module = compile_batch(threads, o.dtype, desc, cache_dir_setting(), B->min_blocks);
        compile_cpu += B->module->compile_ms;
        if (B->module->status != CT_OK) return fail(CT_ERR_COMPILE, "%s", B->module->error.c_str());
        if (B->module->smem > smem_limit)
            return fail(CT_ERR_INVALID_CONFIG, "batch kernel needs too much shared memory");
        if ((st = load_variant(*B->module)) != CT_OK) return st;   // also fills in the register count
        // problem table, tensor maps and work list: most expensive tiles first
        // (solo problems keep zeroed entries that no work item names)
        for (int i = 0; i < n; ++i) {
            const int b = B->item_bucket[(size_t)i];
            if (b < 0) {
                probs.push_back(DevProblem{});
                continue;
            }
            probs.push_back(dev_problem(*B, i, b, B->buckets[(size_t)b].cfg));
            alignas(64) unsigned char map[kTensorMapBytes];
            if ((st = item_map(*B, i, B->buckets[(size_t)b].cfg, map)) != CT_OK) return st;
            memcpy(maps.data() + (size_t)i * kTensorMapBytes, map, kTensorMapBytes);
        }
        std::vector<int> border(B->buckets.size());
        std::iota(border.begin(), border.end(), 0);
        auto tile_cost = [&](int b) {
            const auto& k = B->buckets[(size_t)b];
            return (double)k.fw * k.fh * tile_w(threads, k.cfg) * tile_h(threads, k.cfg);
        };
        std::stable_sort(border.begin(), border.end(), [&](int a, int b) { return tile_cost(a) > tile_cost(b); });
        std::vector<size_t> bstart;   // first work item of each bucket, in `border` order
        for (int b : border) {
            bstart.push_back(work.size());
            std::vector<int> its = B->buckets[(size_t)b].items;
            std::stable_sort(its.begin(), its.end(), [&](int a, int c) {
                return (int64_t)items[a].out_w * items[a].out_h > (int64_t)items[c].out_w * items[c].out_h;
            });
            for (int i : its) {
                const TileCfg& c = B->buckets[(size_t)b].cfg;
                if (!tile_grid_ok(items[i].out_w, items[i].out_h, tile_w(threads, c), tile_h(threads, c)))
                    return fail(CT_ERR_UNSUPPORTED, "batch item %d: more than %lld tiles along one side", i,
                                (long long)kMaxTilesPerSide);
                int64_t tx = 0;
                const int64_t nt = tiles_of(items[i], threads, c, &tx);
                for (int64_t k = 0; k < nt; ++k) work.push_back(work_item((uint32_t)i, k, tx, b, B->filt_off[(size_t)i]));
            }
        }
        if (work.size() > (size_t)0x7fffffff) return fail(CT_ERR_UNSUPPORTED, "too many tiles in one batch");
        // second order: the buckets interleaved, each advancing through its own
        // items at the same relative rate (item j of a bucket of m at (j + 1/2) / m),
        // so tiles bound by memory bandwidth (small filters) run beside tiles bound
        // by the FMA pipe (large filters) instead of after them
        bstart.push_back(work.size());
        std::vector<std::pair<double, size_t>> key;
        key.reserve(work.size());
        for (size_t q = 0; q + 1 < bstart.size(); ++q) {
            const size_t m = bstart[q + 1] - bstart[q];
            for (size_t j = 0; j < m; ++j) key.emplace_back(((double)j + 0.5) / (double)m, bstart[q] + j);
        }
        std::stable_sort(key.begin(), key.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        const size_t nw = work.size();
        for (size_t j = 0; j < nw; ++j) work.push_back(work[key[j].second]);
    }
    B->n_work = (int64_t)(work.size() / 2);
    if ((e = cudaMalloc((void**)&B->d_counter, kCounterWords * sizeof(unsigned))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(batch counter)");
    cudaMemsetAsync(B->d_counter, 0, kCounterWords * sizeof(unsigned), s);
    if (persistent) {
        if ((e = cudaMalloc(&B->d_probs, probs.size() * sizeof(DevProblem))) != cudaSuccess ||
            (e = cudaMalloc(&B->d_work, std::max<size_t>(1, work.size()) * sizeof(WorkItem))) != cudaSuccess ||
            (e = cudaMalloc(&B->d_tmaps, maps.size())) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(batch tables)");
        cudaMemcpyAsync(B->d_probs, probs.data(), probs.size() * sizeof(DevProblem), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(B->d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, s);
        if (!work.empty())
            cudaMemcpyAsync(B->d_work, work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
        B->grid = occupancy_grid(*B->module, threads, o.blocks_per_sm, std::max<int64_t>(1, B->n_work));
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "upload batch tables");
    if (!device_error_word()) return fail(CT_ERR_CUDA, "no device error word");   // allocated before capture
    // capture: the solo launches spread round-robin over forked streams (their
    // ramps and tails overlap, small ones run side by side), then counter
    // reset + the persistent launch, either after all solo launches (joined)
    // or on a branch of its own beside them (`beside`; its blocks then take
    // SMs as the solo launches leave them).  The fork streams and events live
    // only for the capture.
    const size_t nfs = std::min<size_t>(o.solo_branches > 0 ? (size_t)o.solo_branches : 12, B->solo_items.size());
    struct Forks {
        std::vector<cudaStream_t> streams;
        std::vector<cudaEvent_t> events;
        ~Forks()
        {
            for (auto x : streams) cudaStreamDestroy(x);
            for (auto x : events) cudaEventDestroy(x);
        }
    } forks;
    for (size_t k = 0; k < nfs + 2; ++k) {
        cudaEvent_t ev = nullptr;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
        forks.events.push_back(ev);
    }
    for (size_t k = 0; k < nfs + 1; ++k) {
        cudaStream_t x = nullptr;
        if ((e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
        forks.streams.push_back(x);
    }
    auto capture = [&](const std::vector<VariantPtr>& vars, bool beside, int order,
                       cudaGraphExec_t* exec) -> ct_status {
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamBeginCapture");
        ct_status cst = CT_OK;
        if (nfs > 0 || (beside && persistent)) cudaEventRecord(forks.events[0], s);
        for (size_t k = 0; k < nfs; ++k) cudaStreamWaitEvent(forks.streams[k], forks.events[0], 0);
        auto persistent_launch = [&](cudaStream_t ps) {
            const WorkItem* wl = static_cast<const WorkItem*>(B->d_work) + (order ? B->n_work : 0);
            DevParams prm{B->d_probs, wl, B->d_filters, B->d_tmaps, B->d_counter, (int32_t)B->n_work, 0};
            cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned), ps);
            return launch_batch(*B->module, B->grid, threads, prm, ps);
        };
        if (beside && persistent) {
            cudaStream_t ps = forks.streams[nfs];
            cudaStreamWaitEvent(ps, forks.events[0], 0);
            cst = persistent_launch(ps);
        }
        for (size_t k = 0; k < B->solo_items.size() && cst == CT_OK; ++k) {
            const ct_batch_item& it = items[B->solo_items[k]];
            const ct_problem p{it.out_w, it.out_h, it.filter_w, it.filter_h, it.in_pitch, it.out_pitch, o.dtype, 0};
            // one block per tile: the solo launches run beside each other, and
            // small blocks let the hardware interleave them
            cst = launch_variant(*vars[k], p, it.d_image, it.h_filter, it.d_out, forks.streams[k % nfs], 0);
        }
        for (size_t k = 0; k < nfs; ++k) {
            cudaEventRecord(forks.events[k + 1], forks.streams[k]);
            cudaStreamWaitEvent(s, forks.events[k + 1], 0);
        }
        if (beside && persistent) {
            cudaEventRecord(forks.events[nfs + 1], forks.streams[nfs]);
            cudaStreamWaitEvent(s, forks.events[nfs + 1], 0);
        }
        if (cst == CT_OK && persistent && !beside) cst = persistent_launch(s);
        ce = cudaStreamEndCapture(s, &g);
        if (cst != CT_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return cst != CT_OK ? cst : cuda_fail(ce, "cudaStreamEndCapture");
        }
        ce = cudaGraphInstantiate(exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
        return CT_OK;
    };
    // Candidate graphs: solo launches in the tuned forms, and (when some won
    // in the paired multiply-add form, which is faster alone but may overlap
    // worse with its neighbours) with their scalar twins; each with the
    // persistent launch after the solo launches and, when the plan has both,
    // beside them; each with the persistent launch taking its work bucket by
    // bucket or interleaved (when it has more than one bucket).  With more
    // than one candidate, all are timed (replays, interleaved, median of 5
    // after 2 warm-ups; this writes every output) and the fastest is kept.
    std::vector<VariantPtr> scalar = B->solo_vars;
    bool any_pair = false;
    for (size_t k = 0; k < scalar.size(); ++k) {
        if (!scalar[k]->key.cfg.fma2) continue;
        any_pair = true;
        VariantKey sk = scalar[k]->key;
        sk.cfg.fma2 = 0;
        VariantPtr v = get_variant(sk);
        if (!v || v->status != CT_OK || (st = load_variant(*v)) != CT_OK)
            return fail(CT_ERR_COMPILE, "scalar twin of a solo variant: %s", v ? v->error.c_str() : "none");
        scalar[k] = v;
    }
    struct Cand {
        const std::vector<VariantPtr>* vars;
        bool beside;
        int order;
        cudaGraphExec_t exec = nullptr;
        std::vector<float> ms;
    };
    std::vector<Cand> cands;
    const int n_orders = persistent && B->buckets.size() > 1 ? 2 : 1;
    for (int form = 0; form < (any_pair ? 2 : 1); ++form)
        for (int beside = 0; beside < (persistent && nfs > 0 ? 2 : 1); ++beside) {
            if ((o.persistent_layout == 1 && beside) || (o.persistent_layout == 2 && !beside && nfs > 0 && persistent))
                continue;
            for (int order = 0; order < n_orders; ++order) {
                if ((o.work_order == 1 && order) || (o.work_order == 2 && !order && n_orders > 1)) continue;
                cands.push_back(Cand{form ? &scalar : &B->solo_vars, beside != 0, order});
            }
        }
    auto drop = [&]() {
        for (auto& c : cands)
            if (c.exec) cudaGraphExecDestroy(c.exec);
    };
    for (auto& c : cands)
        if ((st = capture(*c.vars, c.beside, c.order, &c.exec)) != CT_OK) {
            drop();
            return st;
        }
    size_t keep = 0;
    if (cands.size() > 1) {
        std::vector<cudaEvent_t> ev(cands.size() + 1);
        for (auto& x : ev) cudaEventCreate(&x);
        e = cudaSuccess;
        for (int r = 0; r < 7 && e == cudaSuccess; ++r) {
            cudaEventRecord(ev[0], s);
            for (size_t c = 0; c < cands.size(); ++c) {
                cudaGraphLaunch(cands[c].exec, s);
                cudaEventRecord(ev[c + 1], s);
            }
            if ((e = cudaEventSynchronize(ev[cands.size()])) != cudaSuccess) break;
            for (size_t c = 0; c < cands.size() && r >= 2; ++c) {
                float x = 0.f;
                cudaEventElapsedTime(&x, ev[c], ev[c + 1]);
                cands[c].ms.push_back(x);
            }
        }
        for (auto& x : ev) cudaEventDestroy(x);
        if (e != cudaSuccess) {
            drop();
            return cuda_fail(e, "timing the batch graph forms");
        }
        double best = INFINITY;
        for (size_t c = 0; c < cands.size(); ++c) {
            std::sort(cands[c].ms.begin(), cands[c].ms.end());
            const double med = cands[c].ms[cands[c].ms.size() / 2];
            if (med < best) {
                best = med;
                keep = c;
            }
        }
    }
    B->exec = cands[keep].exec;
    cands[keep].exec = nullptr;
    if (cands[keep].vars == &scalar) B->solo_vars = scalar;
    B->info.persistent_beside = cands[keep].beside ? 1 : 0;
    B->info.work_interleaved = cands[keep].order;
    drop();
    for (const auto& v : B->solo_vars) B->info.n_solo_fma2 += v->key.cfg.fma2 ? 1 : 0;
    B->info.n_items = n;
    B->info.n_buckets = (int32_t)B->buckets.size();
    B->info.n_work = B->n_work;
    B->info.grid = B->grid;
    B->info.threads = threads;
    B->info.smem_bytes = persistent ? (int32_t)B->module->smem : 0;
    B->info.regs = persistent ? B->module->regs : 0;
    B->info.compile_cpu_ms = compile_cpu;
    B->info.n_solo = (int32_t)B->solo_items.size();
    B->info.plan_ms = now_ms() - t0;
    *out = B.release();
    return CT_OK;
}

CT_API ct_status ct_batch_run(ct_batch* b, void* stream)
{
    if (!b || !b->exec) return fail(CT_ERR_INVALID_ARG, "batch is NULL");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(batch)");
    return CT_OK;
}

CT_API ct_status ct_batch_check(const ct_batch* b)
{
    if (!b || !b->d_counter) return fail(CT_ERR_INVALID_ARG, "batch is NULL");
    unsigned words[kCounterWords] = {};
    const cudaError_t e = cudaMemcpy(words, b->d_counter, sizeof words, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read the batch status");
    if (words[1] & 1u) return fail(CT_ERR_TIMEOUT, "a block of an earlier run gave up waiting for its input copies");
    if (!b->solo_items.empty()) {
        unsigned* w = device_error_word();
        unsigned dw = 0;
        if (w && cudaMemcpy(&dw, w, 4, cudaMemcpyDeviceToHost) == cudaSuccess && (dw & 1u))
            return fail(CT_ERR_TIMEOUT, "a single-problem launch on this device gave up waiting for its input copy");
        cudaGetLastError();
    }
    return CT_OK;
}

CT_API ct_status ct_batch_info_get(const ct_batch* b, ct_batch_info* out)
{
    if (!b || !out) return fail(CT_ERR_INVALID_ARG, "batch and out must be non-NULL");
    *out = b->info;
    return CT_OK;
}

CT_API ct_status ct_batch_bucket(const ct_batch* b, int32_t k, int32_t* filter_w, int32_t* filter_h,
                                 int32_t* n_items, ct_bucket_config* cfg, double* pp)
{
    if (!b) return fail(CT_ERR_INVALID_ARG, "batch is NULL");
    if (k < 0 || k >= (int32_t)b->buckets.size()) return fail(CT_ERR_INVALID_ARG, "bucket %d out of range", k);
    const auto& bk = b->buckets[(size_t)k];
    if (filter_w) *filter_w = bk.fw;
    if (filter_h) *filter_h = bk.fh;
    if (n_items) *n_items = (int32_t)bk.items.size();
    if (cfg) *cfg = ct_bucket_config{bk.cfg.bx, b->threads / bk.cfg.bx, bk.cfg.tx, bk.cfg.ty, bk.cfg.un, bk.cfg.p2};
    if (pp) *pp = bk.pp;
    return CT_OK;
}

CT_API int32_t ct_batch_item_bucket(const ct_batch* b, int32_t i)
{
    if (!b || i < 0 || i >= (int32_t)b->item_bucket.size()) return -1;
    return b->item_bucket[(size_t)i];
}

CT_API void ct_batch_free(ct_batch* b) { delete b; }

}  // extern "C"
