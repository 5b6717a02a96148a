// Internal pieces of the persistent batched kernel shared by the planned
// batch (batch.cpp) and the request server (serve.cpp).
#pragma once

#include "ct_internal.hpp"

#include <algorithm>
#include <string>
#include <vector>

namespace ct {

struct TileCfg {
    int bx = 32, tx = 4, ty = 4, un = 0;
};

// Mirrors of the device structs in batch.cuh.
struct DevProblem {
    const void* in;
    float* out;
    int64_t in_pitch, out_pitch;
    int32_t out_w, out_h, in_w, in_h;
    int32_t bucket, tiles_x, filt_off, pad;
};
static_assert(sizeof(DevProblem) == 64, "DevProblem layout");
struct DevParams {
    const void* probs;
    const void* work;
    const float* filters;
    unsigned* counter;
    int32_t n_work;
    int32_t pad;
};
static_assert(sizeof(DevParams) == 40, "DevParams layout");
struct WorkItem {
    uint32_t problem, tile;
};

constexpr int64_t kSmemPerSM = 233472;   // shared memory per SM usable by blocks
constexpr int kMinBlocks = 4;            // resident blocks per SM the batch kernel is built for

struct BucketDesc {
    int fw, fh;
    TileCfg cfg;
};

inline int64_t tile_w(int threads, const TileCfg& c) { (void)threads; return (int64_t)c.bx * c.tx; }
inline int64_t tile_h(int threads, const TileCfg& c) { return (int64_t)(threads / c.bx) * c.ty; }

// floats of one item buffer (taps + halo), a multiple of 4
inline int64_t bucket_buf_floats(int threads, const TileCfg& c, int fw, int fh)
{
    const int64_t hh = tile_h(threads, c) + fh - 1;
    const int64_t sw = round_up(tile_w(threads, c) + fw - 1, 4);
    return round_up(fh * round_up(fw, 4) + hh * sw, 4);
}

// dynamic shared memory of the kernel: two item buffers
inline int64_t bucket_smem(int threads, const TileCfg& c, int fw, int fh)
{
    return 2 * 4 * bucket_buf_floats(threads, c, fw, fh);
}

std::vector<std::string> batch_options(int threads, int dtype, const std::vector<BucketDesc>& b);

uint64_t options_key(const std::vector<std::string>& o);

VariantPtr compile_batch(int threads, int dtype, const std::vector<BucketDesc>& b, const std::string& dir);

ct_status launch_batch(Variant& v, int grid, int threads, const DevParams& prm, cudaStream_t s);

int occupancy_grid(Variant& v, int threads, int blocks_per_sm, int64_t n_work);


}  // namespace ct
