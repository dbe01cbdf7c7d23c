// seeds_device.cuh -- device-side data layout of the SEEDS GB300 path.
//
// One DevImage per image of a context, resident in device memory.  The
// persistent kernel walks a host-built schedule: a list of steps, each step
// a list of (image, op) entries whose work is flattened into one range of
// "virtual threads" (every entry padded to a multiple of 32 so that a warp
// never straddles two entries).  A step is an evaluate slot, a grid
// barrier, and -- when the step holds a phase -- an apply slot and another
// barrier.
#pragma once

#include <cstdint>

#include "seeds.h"

namespace seeds {

constexpr int kMaxLevels = SEEDS_MAX_LEVELS;
constexpr uint16_t kNoLabel = 0xFFFF;  // labels are < 65535

// op kinds (same numbering as the debug hooks of seeds.h)
enum : int32_t { OP_INIT = 0, OP_PHASE = 1, OP_DESCEND = 2, OP_OUTPUT = 3 };

// device error word bits
enum : int32_t { DERR_TIMEOUT = 1, DERR_BOUNDS = 2, DERR_INJECTED = 4 };

struct DevImage {
    // geometry and parameters
    int32_t W, H, K, gx, gy, L, iters, B, nbins, patch, gnum, gden;
    int32_t bins16;       // bin map stored as uint16 (B^3 > 256)
    int32_t hist_jmajor;  // hist[j*K + k] instead of hist[k*nbins + j]
    int32_t nbx[kMaxLevels + 1], nby[kMaxLevels + 1];  // level 0 = W, H
    int32_t group[kMaxLevels + 1];                     // lanes per unit (1 or 32)
    const int32_t *xe[kMaxLevels + 1];                 // block column edges, level >= 1
    const int32_t *ye[kMaxLevels + 1];                 // block row edges, level >= 1
    // state
    void *bins;                      // colour bin per pixel
    uint16_t *lab[kMaxLevels + 1];   // lab[0]: pixel labels; lab[l]: level-l block grid
    int32_t *hist;                   // K x nbins counts
    int32_t *size;                   // |A_k|
    uint32_t *moves;                 // 2 words per accepted move of the current phase
    int32_t moves_cap;
    int32_t *cnt;                    // 2 move counters (step parity)
    // per call
    const uint8_t *rgb;
    int64_t stride;
    int32_t *out;
};

struct StepEntry {
    int32_t img;
    int32_t op;
    int32_t level;
    int32_t phase;
    int64_t vt_begin;  // first virtual thread of the entry inside its step
    int32_t units;     // units of work (threads or warps, see group)
    int32_t group;     // 1: one thread per unit, 32: one warp per unit
};

struct Schedule {
    const StepEntry *ent;
    const int32_t *step_first;  // nsteps + 1
    const int64_t *step_vt;     // virtual threads of each step
    const int32_t *step_apply;  // step has a phase entry
    int32_t nsteps;
    int32_t max_nbins;          // largest histogram of the context (scratch size)
    unsigned long long *trace;  // optional: 1 + 2*nsteps globaltimer stamps
};

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

struct IoEntry {
    const uint8_t *rgb;
    int64_t stride;
    int32_t *out;
};

constexpr int kIoChunk = 64;
struct IoChunk {
    int32_t first, n;
    IoEntry e[kIoChunk];
};

// per-warp shared-memory scratch for a bin count of `nbins`:
//   int32[4]       header; [0] = number of distinct bins listed
//   int32[nbins]   histogram (kept all-zero between uses)
//   uint16[nbins]  the distinct bins seen
constexpr int kScratchHeader = 4;
__host__ __device__ inline int warp_scratch_bytes(int nbins)
{
    int b = kScratchHeader * 4 + nbins * 4 + nbins * 2;
    return (b + 15) & ~15;
}

// launch helpers (seeds_kernels.cu)
cudaError_t launch_set_io(DevImage *d_imgs, const IoChunk &chunk, cudaStream_t s);
cudaError_t launch_persistent(const DevImage *d_imgs, const Schedule &sch, GridBarrier *bar, int32_t *err,
                              int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t persistent_max_blocks_per_sm(int threads, size_t smem, int *n);
cudaError_t prepare_persistent(size_t smem);
cudaError_t launch_recount(const DevImage *d_imgs, int img, int level, int64_t npix, cudaStream_t s);

}  // namespace seeds
