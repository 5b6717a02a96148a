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
    int p2 = 0;   // 1: paired multiply-adds over output-row pairs (needs un = 1 and an even ty)
};

// Mirrors of the device structs in batch.cuh.
struct DevProblem {
    const void* in;
    float* out;
    int64_t in_pitch, out_pitch;
    int32_t out_w, out_h, in_w, in_h;
    int32_t bucket, tiles_x, filt_off, pad;   // tiles_x is for inspection: work items carry their tile
};
static_assert(sizeof(DevProblem) == 64, "DevProblem layout");
struct DevParams {
    const void* probs;
    const void* work;
    const float* filters;
    const void* tmaps;   // one 128-byte tensor map per problem
    unsigned* counter;   // kCounterWords words: next work item, error bits
    int32_t n_work;
    int32_t pad;
};
static_assert(sizeof(DevParams) == 48, "DevParams layout");
constexpr int kCounterWords = 2;
// One tile of one problem; the tile is (row << 16) | column, so the kernel
// places it without a division.  The record also carries the problem's
// bucket and filter offset, so a block stages and dispatches an item after
// one 16-byte load.
struct WorkItem {
    uint32_t problem, tile, bucket, filt_off;
};
static_assert(sizeof(WorkItem) == 16, "WorkItem layout");
constexpr int64_t kMaxTilesPerSide = 65535;
inline WorkItem work_item(uint32_t problem, int64_t k, int64_t tiles_x, int32_t bucket, int32_t filt_off)
{
    return WorkItem{problem, (uint32_t)(((k / tiles_x) << 16) | (k % tiles_x)), (uint32_t)bucket,
                    (uint32_t)filt_off};
}
inline bool tile_grid_ok(int64_t out_w, int64_t out_h, int64_t tw, int64_t th)
{
    return (out_w + tw - 1) / tw <= kMaxTilesPerSide && (out_h + th - 1) / th <= kMaxTilesPerSide;
}

constexpr int64_t kSmemPerSM = 233472;   // shared memory per SM usable by blocks
constexpr int kMinBlocks = 4;            // resident blocks per SM the batch kernel is built for

struct BucketDesc {
    int fw, fh;
    TileCfg cfg;
};

inline int64_t tile_w(int threads, const TileCfg& c) { (void)threads; return (int64_t)c.bx * c.tx; }
inline int64_t tile_h(int threads, const TileCfg& c) { return (int64_t)(threads / c.bx) * c.ty; }

// The halo box of a tile: the tile plus the filter's apron, its width rounded
// up to 16 bytes; at most 256 elements per side (the tensor-copy limit).
inline int64_t batch_box_w(int threads, const TileCfg& c, int fw, int dtype)
{
    return round_up(tile_w(threads, c) + fw - 1, 16 / elem_size(dtype));
}
inline int64_t batch_box_h(int threads, const TileCfg& c, int fh) { return tile_h(threads, c) + fh - 1; }
inline bool halo_box_ok(int threads, const TileCfg& c, int fw, int fh, int dtype)
{
    return batch_box_w(threads, c, fw, dtype) <= 256 && batch_box_h(threads, c, fh) <= 256 &&
           tile_w(threads, c) % 16 == 0;
}

// Floats of one filter in the batch's filter table: fh rows of taps padded
// to a multiple of 4, then fh - 1 rows of (f[i][j], f[i-1][j]) pairs padded
// to an even count (read by buckets in the paired form).  Both parts are
// multiples of 4 floats, so every filter starts on a 16-byte boundary.
inline int64_t filter_rows_floats(int fw, int fh) { return (int64_t)fh * round_up(fw, 4); }
inline int64_t filter_pairs_floats(int fw, int fh) { return (int64_t)(fh - 1) * round_up(fw, 2) * 2; }

// Appends one FP32 filter (fh x fw, row-major) to a batch filter table in the
// layout above; returns its offset in floats.
inline int64_t append_filter(std::vector<float>& table, const float* f, int fw, int fh)
{
    const int64_t off = (int64_t)table.size();
    const int fwp = (int)round_up(fw, 4), fwp2 = (int)round_up(fw, 2);
    for (int i = 0; i < fh; ++i)
        for (int j = 0; j < fwp; ++j) table.push_back(j < fw ? f[i * fw + j] : 0.0f);
    for (int i = 1; i < fh; ++i)
        for (int j = 0; j < fwp2; ++j) {
            table.push_back(j < fw ? f[i * fw + j] : 0.0f);
            table.push_back(j < fw ? f[(i - 1) * fw + j] : 0.0f);
        }
    return off;
}

// Whether a bucket tile can take the paired form.
inline bool pair_ok(const TileCfg& c) { return c.un == 1 && c.ty >= 2 && c.ty % 2 == 0; }

// bytes of one item buffer (halo box, then taps and, paired, tap pairs), a multiple of 128
inline int64_t bucket_buf_bytes(int threads, const TileCfg& c, int fw, int fh, int dtype)
{
    const int64_t halo = batch_box_w(threads, c, fw, dtype) * batch_box_h(threads, c, fh) * elem_size(dtype);
    const int64_t taps = 4 * (filter_rows_floats(fw, fh) + (c.p2 ? filter_pairs_floats(fw, fh) : 0));
    return round_up(round_up(halo, 16) + taps, 128);
}

// dynamic shared memory of the kernel: two item buffers plus alignment slack
inline int64_t bucket_smem(int threads, const TileCfg& c, int fw, int fh, int dtype)
{
    return 2 * bucket_buf_bytes(threads, c, fw, fh, dtype) + 128;
}

// min_blocks: resident blocks per SM the register allocation must allow
// (__launch_bounds__ minimum), kMinBlocks unless a plan asks otherwise.
std::vector<std::string> batch_options(int threads, int dtype, const std::vector<BucketDesc>& b,
                                       int min_blocks = kMinBlocks);

uint64_t options_key(const std::vector<std::string>& o);

VariantPtr compile_batch(int threads, int dtype, const std::vector<BucketDesc>& b, const std::string& dir,
                         int min_blocks = kMinBlocks);

ct_status launch_batch(Variant& v, int grid, int threads, const DevParams& prm, cudaStream_t s);

int occupancy_grid(Variant& v, int threads, int blocks_per_sm, int64_t n_work);


}  // namespace ct
