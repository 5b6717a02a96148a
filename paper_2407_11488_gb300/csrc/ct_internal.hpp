// Internal declarations shared by the convtune host library translation units.
#pragma once

#include "convtune.h"

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <future>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

struct ct_space;
struct ct_table;

namespace ct {

// ---------------------------------------------------------------- errors ---
void set_error(const std::string& msg);
void clear_error();
ct_status fail(ct_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
ct_status cuda_fail(cudaError_t e, const char* what);

// --------------------------------------------------------------- problem ---
constexpr int kDefaultSmemLimit = 232448;   // GB300 opt-in shared memory per block
constexpr int kMaxThreads = 1024;
constexpr int kMaxTile = 16;

inline int elem_size(int dtype) { return dtype == CT_BF16 ? 2 : 4; }
inline int64_t in_w(const ct_problem& p) { return (int64_t)p.out_w + p.filter_w - 1; }
inline int64_t in_h(const ct_problem& p) { return (int64_t)p.out_h + p.filter_h - 1; }
inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Problem ranges and pitches (not pointers).
ct_status check_problem(const ct_problem* p);
// Config ranges and launchability for p (smem_limit <= 0: device or default).
ct_status check_config(const ct_problem& p, const ct_config& c, int smem_limit);
int64_t smem_bytes(const ct_problem& p, const ct_config& c);
int device_smem_limit();   // current device's opt-in limit, else the default
double problem_flops(const ct_problem& p);

// ------------------------------------------------------------------ rng ----
// SplitMix64 in counter form: draw i of stream seed = mix(seed + (i+1)*gamma).
uint64_t splitmix64_at(uint64_t seed, uint64_t i);
struct Rng {
    uint64_t seed, i = 0;
    explicit Rng(uint64_t s) : seed(s) {}
    uint64_t next() { return splitmix64_at(seed, i++); }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    uint64_t below(uint64_t n) { return n ? next() % n : 0; }
};

// ---------------------------------------------------------------- spaces ---
struct Space {
    // Fixed parameter order: block_x, block_y, tile_x, tile_y, use_smem, unroll.
    std::vector<int> vals[6];
    std::string name;
    int64_t raw_size() const;
    ct_config at(int64_t canonical) const;
    int64_t index_of(const ct_config& c) const;   // -1 if not a point of the space
};
extern const char* const kParamNames[6];
inline int cfg_get(const ct_config& c, int k) {
    const int32_t* v = &c.block_x;
    return v[k];
}
inline void cfg_set(ct_config& c, int k, int v) {
    int32_t* p = &c.block_x;
    p[k] = v;
}

struct Entry {
    int64_t index;
    ct_config cfg;
};
std::vector<Entry> enumerate_valid(const Space& s, const ct_problem& p, int smem_limit);

// -------------------------------------------------------------- variants ---
struct VariantKey {
    ct_config cfg;
    int fw, fh, dtype;
    // non-empty: the taps (FP32, fh x fw) compiled into the variant as immediates
    std::vector<float> taps;
    uint64_t packed() const;
    std::string describe() const;
};
// The key of the variant that runs (p, c) with filter h_filter: the taps are
// part of it when c.taps = 1, c.unroll = 1 and every tap is finite.
VariantKey variant_key(const ct_problem& p, const ct_config& c, const void* h_filter);

struct Variant {
    VariantKey key{};
    std::string kname = "ct_corr2d";
    std::vector<char> cubin;
    std::string log;
    int status = CT_OK;
    std::string error;
    int regs = 0, spill_bytes = 0;
    int64_t smem = 0;
    double compile_ms = 0.0;
    bool from_cache = false;
    // loaded state (guarded by mu)
    std::mutex mu;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    int loaded_device = -1;
    int64_t smem_attr = -1;
    int resident = 0;   // blocks the loaded device holds at once (SMs x blocks per SM), 0 until loaded
    ~Variant();
};
using VariantPtr = std::shared_ptr<Variant>;

// Writes the 128-byte tensor map (64-byte aligned `map`) of an image of
// in_w x in_h elements, rows in_pitch elements apart, 16-byte aligned, whose
// box (box_w x box_h elements, each at most 256, box_w a multiple of 16 bytes)
// is the halo of one tile; elements outside the image read as zero.
ct_status encode_halo_map(void* map, const void* d_image, int dtype, int64_t in_w, int64_t in_h, int64_t in_pitch,
                          int64_t box_w, int64_t box_h);
constexpr size_t kTensorMapBytes = 128;

// The single-problem kernel stages its halo with one tensor copy when it uses
// shared memory and the halo box fits (at most 256 x 256 elements).
int64_t halo_box_w(const ct_config& c, int fw, int dtype);
int64_t halo_box_h(const ct_config& c, int fh);
bool tma_staged(const ct_config& c, int fw, int fh, int dtype);
// Device word whose bit 0 the kernels set when a bounded wait gave up
// (allocated on first use on each device; NULL without a device).
unsigned* device_error_word();
// Reads the current device's error word (synchronously) and clears it;
// true when bit 0 was set.
bool take_device_error();

// Compiles with NVRTC, consulting the on-disk cache (thread safe; no device needed).
VariantPtr compile_variant(const VariantKey& k, const std::string& cache_dir);
VariantPtr compile_source(const char* src, size_t len, const char* prog_name, const std::vector<std::string>& opts,
                          const std::string& kernel_name, const std::string& cache_dir);
std::vector<std::string> nvrtc_base_options();
void add_env_options(std::vector<std::string>& o);
// Library-wide in-memory cache on top of compile_variant.
VariantPtr get_variant(const VariantKey& k);
void put_variant(const VariantPtr& v);
void clear_variants();
std::string& cache_dir_setting();

ct_status load_variant(Variant& v);
void unload_variant(Variant& v);

// Builds the parameter block and launches one correlation; persist selects
// the grid (one block per tile, or the persistent grid of v.resident blocks).
ct_status launch_variant(Variant& v, const ct_problem& p, const void* d_image,
                         const void* h_filter, float* d_out, cudaStream_t stream, int persist = 0);
// Output tiles of p under configuration c.
int64_t tile_count(const ct_problem& p, const ct_config& c);
// Pointer and layout checks for a launch (alignment, non-null).
ct_status check_buffers(const ct_problem& p, const void* d_image, const void* h_filter, const float* d_out);
ct_status require_device();

// ------------------------------------------------------------ aux kernels ---
// Seeded uniform[-1,1) fill of a pitched float or bf16 image (device side).
cudaError_t launch_fill_uniform(void* dst, int dtype, int64_t rows, int64_t cols, int64_t pitch,
                                uint64_t seed, uint64_t start, cudaStream_t s);
cudaError_t launch_l2_flush(void* buf, int64_t bytes, uint32_t salt, cudaStream_t s);

// ----------------------------------------------------------- compile pool ---
class CompilePool {
public:
    using Job = std::function<VariantPtr()>;
    // reserve_urgent threads are kept for urgent requests: speculative jobs
    // run on at most threads - reserve_urgent of them at a time.
    CompilePool(int nthreads, std::string cache_dir, int reserve_urgent = 0);
    ~CompilePool();
    // urgent requests go to the front of the queue (or move there if queued)
    std::shared_future<VariantPtr> request(const VariantKey& k, bool urgent = false);
    std::shared_future<VariantPtr> request(uint64_t key, Job job, bool urgent = false);
    void forget(const VariantKey& k);
    void forget(uint64_t key);
    // true when the job for k has finished, or is not in the pool
    bool ready(const VariantKey& k);
    const std::string& cache_dir() const { return cache_dir_; }
    size_t queued();
    size_t threads() const { return threads_.size(); }
private:
    struct Item {
        uint64_t key;
        Job job;
        std::shared_ptr<std::promise<VariantPtr>> pr;
        bool urgent = false;
    };
    void worker();
    std::string cache_dir_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<Item> queue_;
    std::unordered_map<uint64_t, std::shared_future<VariantPtr>> futures_;
    std::vector<std::thread> threads_;
    size_t max_speculative_ = 0, running_speculative_ = 0;
    bool stop_ = false;
};

double now_ms();
const char* last_error();
// Current device's SM clock in MHz, read through NVML (0 when unavailable).
int sample_sm_mhz();

ct_status tune_gpu(const ct_problem* p, const ct_space* s, ct_strategy st, const ct_tune_opts* opts,
                   const void* d_image, const void* h_filter, float* d_out, ct_config* best_out,
                   ct_table** table_out);
ct_status tune_replay(const ct_problem* p, const ct_space* s, ct_strategy st, const ct_tune_opts* opts,
                      const double* times, int64_t n_times, ct_config* best_out, ct_table** table_out);
ct_status write_table(const ct_table& t, const char* path, const std::string& tag, bool append);
bool builtin_space(const char* name, Space& s);
bool space_from_json(const char* js, Space& s, std::string& err);

}  // namespace ct

// Opaque handles of the C-ABI.
struct ct_space {
    ct::Space s;
};
struct ct_table {
    std::vector<ct_row> rows;
    ct_table_info info{};
    std::string tag;   // problem description written with every JSONL row
};
