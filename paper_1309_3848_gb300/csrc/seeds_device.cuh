// seeds_device.cuh -- device-side data layout and op schedule of the SEEDS
// GB300 path.
//
// One DevImage per image, resident in device memory.  The persistent kernel
// walks a schedule: a list of steps, each step a list of entries whose work
// is flattened into one range of "virtual threads" (every entry padded to a
// multiple of 32 so that a warp never straddles two entries), followed by
// one grid barrier.
//
// State is double-buffered.  Op number o of an image reads buffer o&1 of its
// labels, histograms and sizes, and writes the other buffer: its own accepted
// moves go there at once, and so do (a "catch-up" entry of the same step) the
// moves of op o-1, which were applied to buffer o&1 one step earlier.  So
// after ops [0, e) the complete state is in buffer e&1, decisions of a phase
// only ever see the state at phase start, and one barrier per step suffices.
#pragma once

#include <cstdint>

#include "seeds.h"

namespace seeds {

constexpr int kMaxLevels = SEEDS_MAX_LEVELS;
constexpr uint16_t kNoLabel = 0xFFFF;   // labels are < 65535
constexpr uint32_t kNoMove = 0xFFFFFFFFu;

// op kinds (as in the debug hooks of seeds.h); OP_MINIT and OP_MPHASE are
// the start and the phases of the means-based pixel iterations (Sec. 6.5).
// OP_CATCHUP and OP_BTILE occur only in step entries: a catch-up replays the
// previous phase's moves, and OP_BTILE is a block phase (OP_PHASE, level >=
// 1, blocks judged by a warp) run in warp tiles.
enum : int32_t {
    OP_INIT = 0,
    OP_PHASE = 1,
    OP_DESCEND = 2,
    OP_OUTPUT = 3,
    OP_CATCHUP = 4,
    OP_MINIT = 5,
    OP_MPHASE = 6,
    OP_BTILE = 7
};

__host__ __device__ inline bool is_phase(int kind) { return kind == OP_PHASE || kind == OP_MPHASE; }

// device error word bits
enum : int32_t { DERR_TIMEOUT = 1, DERR_BOUNDS = 2, DERR_INJECTED = 4 };

struct DevImage {
    // geometry and parameters
    int32_t W, H, K, gx, gy, L, iters, B, nbins, patch, gnum, gden;
    int32_t bins16;       // bin map stored as uint16 (B^3 > 256)
    int32_t hist_jmajor;  // hist[j*K + k] instead of hist[k*nbins + j]
    int32_t hist_sk, hist_sj;  // hist index = k*hist_sk + j*hist_sj (either layout)
    int32_t small_area;   // blocks up to this many pixels are judged by one thread
    int32_t tile_uy;      // unit rows of a pixel-phase warp tile: 2 or kTileUY
    int32_t color;        // 0: RGB bytes, 1: 8-bit CIE L*a*b* codes (Sec. 6.2)
    int32_t means_iters;  // means-based pixel iterations after the histogram ones
    float means_w;        // (m/S)^2 = m^2 K / N, the spatial weight of SLIC's distance
    int32_t edge_tau;     // edge snapping threshold (Sec. 6.4), 0 = off
    int32_t prior;        // the compactness prior (Sec. 6.4) in the histogram pixel phases
    float compact_w;      // its weight of d^2: (compact_prior/16) * 81 * K / N
    float gamma_f;        // gamma as a float (0 without patches), for the prior's score
    int32_t nbx[kMaxLevels + 1], nby[kMaxLevels + 1];  // level 0 = W, H
    int32_t maxarea[kMaxLevels + 1];                   // largest block of a level
    const int32_t *xe[kMaxLevels + 1];                 // block column edges, level >= 1
    const int32_t *ye[kMaxLevels + 1];                 // block row edges, level >= 1
    // state
    void *bins;                         // colour bin per pixel
    uint16_t *lab[kMaxLevels + 1][2];   // [0]: pixel labels, [l]: level-l block grid; 2 buffers
    int32_t *hist[2];                   // K x nbins counts, 2 buffers
    int32_t *size[2];                   // |A_k|, 2 buffers
    uint32_t *dec[2];                   // per unit of a phase: a move (block: k << 16 | n; histogram pixel phase:
                                        // pixel_dec) or kNoMove; only moves are written, replays reset them
    unsigned long long *msum[2];        // K x 5: sums of the 3 colour codes, of x, of y (means iterations;
                                        // x and y through every move with the compactness prior)
    uint8_t *edges;                     // per pixel, edge snapping: bit 0 across to the right, bit 1 down
    int32_t units_cap;                  // entries of each dec buffer
    int32_t *err;                       // the launch's error word (debug builds report bounds trips here)
    // per call
    const uint8_t *rgb;
    int64_t stride;
    int32_t *out;
};

struct StepEntry {
    int32_t img;
    int32_t op;        // OP_*; OP_CATCHUP replays the moves of op `opidx - 1`
    int32_t level;     // of the op (for a catch-up: of the previous op)
    int32_t phase;
    int32_t opidx;     // the image's op number: selects the buffers
    int32_t units;     // units of work
    int64_t vt_begin;  // first virtual thread of the entry inside its step
    int32_t group;     // 1: one thread per unit, 32: one warp per unit
    int32_t cphase;    // OP_PHASE: the previous phase of the same level, whose
                       // moves the same units replay first; -1 for none
};

struct Schedule {
    const StepEntry *ent;
    const int32_t *step_first;  // nsteps + 1
    const int64_t *step_vt;     // virtual threads of each step
    int32_t nsteps;
    int32_t max_nbins;          // largest histogram of the context (scratch size)
    unsigned long long *trace;  // optional: 1 + nsteps globaltimer stamps
    // anytime termination (Sec. 5.4): stop at the first step boundary after
    // stop_steps steps (> 0) or budget_ns of device time (> 0), write every
    // unfinished image's partition, and store the steps run in *steps_out
    int32_t stop_steps;
    int32_t nimg;
    unsigned long long budget_ns;
    int32_t *steps_out;
    // failure tests: the barrier's time limit (0: 2 s), and a step whose
    // barrier CTA 0 does not arrive at (step + 1; 0: none), so that every
    // wait there runs out and the kernel returns with DERR_TIMEOUT
    unsigned long long timeout_ns;
    int32_t withhold;
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
__host__ __device__ inline int warp_hist_scratch_bytes(int nbins)
{
    int b = kScratchHeader * 4 + nbins * 4 + nbins * 2;
    return (b + 15) & ~15;
}

// The pixel phase works on warp tiles of kTileUX x (2 or kTileUY) units of
// one parity class (a unit per lane and tile row; the row count is a launch
// knob); the warp stages the labels of the tile plus a 2-pixel halo in shared
// memory, behind the histogram scratch, sized here for the taller tile.
constexpr int kTileUX = 32, kTileUY = 4;
constexpr int kTileW = 2 * kTileUX + 4;  // pixel columns staged
__host__ __device__ constexpr int tile_h(int uy) { return 2 * uy + 3; }  // pixel rows staged
constexpr int kTileH = tile_h(kTileUY);
// staged labels, the units' bins, the list of the tile's boundary units
constexpr int kTileBytes = (kTileW * kTileH * 2 + kTileUY * kTileUX * 2 + kTileUY * kTileUX + 15) & ~15;
// A catch-up entry (the replay of a phase's moves on its own) gives a lane
// kCatchupPerLane pixels, a small block a lane each and a block that a warp
// judges a warp each.  In a wide step (kWideStep) a lane takes
// kCatchupPerLane small blocks, and blocks a warp judges of at most
// kCatchupLaneArea pixels take a lane each to read their decisions; the
// warp then replays the moved ones one after another.
constexpr int kCatchupPerLane = 4;
// A warp of a small-block phase takes 32 units of a lattice row, or, on a
// level whose superpixels span at least kSmallTileSpan units per side, a
// kSmallTileX x kSmallTileY block of units: such warps often lie inside
// one superpixel and finish after their ring tests, where a row of 32 units
// always crosses a boundary and runs the judge for its few boundary lanes.
constexpr int kSmallTileX = 8, kSmallTileY = 4, kSmallTileSpan = 16;
constexpr int kCatchupLaneArea = 128;
// descents and the output: cells (pixels) of a row per thread
constexpr int kRowChunk = 8;

__host__ __device__ inline int warp_scratch_bytes(int nbins) { return warp_hist_scratch_bytes(nbins) + kTileBytes; }

// ---------------------------------------------------------------------------
// the op list of one image (shared by the host scheduler and the device-side
// setup of the allocation-free entry point)
// ---------------------------------------------------------------------------

struct OpDesc {
    int32_t kind, level, phase;
};

// init, block levels L..1 (iters*4 phases, then a descent), the pixel level
// (iters*4 phases), with means iterations mi > 0 their start and mi*4
// phases, output
__host__ __device__ inline int num_ops(int L, int iters, int mi)
{
    return 1 + L * (4 * iters + 1) + 4 * iters + (mi > 0 ? 1 + 4 * mi : 0) + 1;
}

__host__ __device__ inline OpDesc op_at(int L, int iters, int mi, int o)
{
    OpDesc d{OP_OUTPUT, 0, 0};
    const int per = 4 * iters + 1, P = 1 + L * per;
    if (o == 0) {
        d.kind = OP_INIT;
    } else if (o < P) {
        const int i = (o - 1) / per, r = (o - 1) % per;
        d.level = L - i;
        if (r < 4 * iters) {
            d.kind = OP_PHASE;
            d.phase = r & 3;
        } else {
            d.kind = OP_DESCEND;
        }
    } else if (o < P + 4 * iters) {
        d.kind = OP_PHASE;
        d.phase = (o - P) & 3;
    } else if (mi > 0 && o == P + 4 * iters) {
        d.kind = OP_MINIT;
    } else if (mi > 0 && o < P + 4 * iters + 1 + 4 * mi) {
        d.kind = OP_MPHASE;
        d.phase = (o - P - 4 * iters - 1) & 3;
    }
    return d;
}

__host__ __device__ inline int64_t phase_units(const DevImage &im, int level, int phase)
{
    return (int64_t)((im.nbx[level] - (phase & 1) + 1) >> 1) * ((im.nby[level] - (phase >> 1) + 1) >> 1);
}

// Threads per unit of a block level: 1 (small blocks, up to small_area
// pixels) or 32 (a warp per block).  A thread sums a block's intersections
// in 32 bits, exact while kSmallMax * W * H < 2^31; larger images give
// every block level to warps.
constexpr int kSmallMax = 16;
__host__ __device__ inline int level_group(const DevImage &im, int level)
{
    if (level == 0) return 1;
    const bool thread = im.maxarea[level] <= im.small_area && (int64_t)im.W * im.H * kSmallMax < (1ll << 31);
    return thread ? 1 : 32;
}

// whether the warps of a small-block phase take 2D blocks of units: the
// superpixels of a level span 2^(L - level) lattice units per side (the
// grid of Sec. 5.1 halves the blocks at each level, the parity lattice takes
// every other block)
__host__ __device__ inline bool small_tiles_2d(const DevImage &im, int level)
{
    return (1 << (im.L - level)) >= kSmallTileSpan;
}

// threads per unit of a catch-up entry, and units per lane where that is 1
__host__ __device__ inline int catchup_group(const DevImage &im, int level, bool wide)
{
    return level > 0 && level_group(im, level) == 32 && (!wide || im.maxarea[level] > kCatchupLaneArea) ? 32 : 1;
}
__host__ __device__ inline int catchup_per_lane(const DevImage &im, int level, bool wide)
{
    return level == 0 || (wide && level_group(im, level) == 1) ? kCatchupPerLane : 1;
}

// The unit lattice of a phase on a grid nx x ny: unit (ux,uy) is cell
// (2ux + px, 2uy + py).  A phase entry that also replays the previous phase
// (cphase >= 0) walks the union of both lattices, so that one thread or warp
// handles unit (ux,uy) of both.
__host__ __device__ inline void lattice(int nx, int ny, int phase, int cphase, int *cols, int *rows)
{
    *cols = (nx - (phase & 1) + 1) >> 1;
    *rows = (ny - (phase >> 1) + 1) >> 1;
    if (cphase >= 0) {
        const int c2 = (nx - (cphase & 1) + 1) >> 1, r2 = (ny - (cphase >> 1) + 1) >> 1;
        *cols = *cols > c2 ? *cols : c2;
        *rows = *rows > r2 ? *rows : r2;
    }
}

// Warp tiles of a block phase are one unit row high.  The warp judges its
// tile's boundary blocks one after another, each a chain of trips to memory,
// so a step is bound by its longest tile; short tiles keep that chain short
// and give the step more warps.
constexpr int kBlockTileUY = 1;

// warp tiles of a phase on a level's grid (level 0: pixels)
__host__ __device__ inline int64_t level_tiles(const DevImage &im, int level, int phase, int cphase)
{
    int cols, rows;
    lattice(im.nbx[level], im.nby[level], phase, cphase, &cols, &rows);
    const int uy = level > 0 ? kBlockTileUY : im.tile_uy;
    return (int64_t)((cols + kTileUX - 1) / kTileUX) * ((rows + uy - 1) / uy);
}

__host__ __device__ inline int64_t pixel_tiles(const DevImage &im, int phase, int cphase)
{
    return level_tiles(im, 0, phase, cphase);
}

// emit_entries' `mode` argument: bits 0-1 the fusion of replays
// (fuse_step), bit 2 a wide step (step_mode): phases of warp-judged blocks
// in warp tiles, catch-ups with more units per lane
constexpr int kWideStep = 4;

// Entries of image `img` for its op `o`.  When the moves of op o-1 (a phase)
// are pending, a phase of the same level replays them unit by unit before
// judging its own units (one fused entry) if `fuse` allows it (2: block and
// pixel phases, 1: pixel phases only, 0: none; see fuse_step); otherwise
// they get a catch-up entry of their own first, whose warps run beside the
// phase's.  The output op needs none: it reads the buffer that the last
// phase wrote its moves into, and nothing reads the other buffer or the
// histograms after it.  Returns the number of entries written; `vt` advances
// by their padded thread counts.
__host__ __device__ inline int emit_entries(const DevImage &im, int img, int o, bool catchup, int mode,
                                            StepEntry *out, int64_t *vt)
{
    const int fuse = mode & 3;
    const bool wide = (mode & kWideStep) != 0;
    int n = 0;
    const OpDesc op = op_at(im.L, im.iters, im.means_iters, o);
    int cphase = -1;
    if (catchup && o > 0 && op.kind != OP_OUTPUT) {
        const OpDesc pv = op_at(im.L, im.iters, im.means_iters, o - 1);
        if (is_phase(pv.kind) && op.kind == pv.kind && pv.level == op.level && fuse >= (op.level == 0 ? 1 : 2)) {
            cphase = pv.phase;
        } else if (is_phase(pv.kind)) {
            const int64_t pu = phase_units(im, pv.level, pv.phase);
            const int group = catchup_group(im, pv.level, wide);
            const int per = catchup_per_lane(im, pv.level, wide);
            const int64_t units = (pu + per - 1) / per;  // lanes (group 1) or warps (group 32)
            const int64_t count = (units * group + 31) / 32 * 32;
            if (count > 0) {
                StepEntry e{img, OP_CATCHUP, pv.level, pv.phase, o, (int32_t)units, *vt, group, -1};
                out[n++] = e;
                *vt += count;
            }
        }
    }
    int64_t units = 0, threads = -1;  // threads: the entry's count when it is not units * group
    int group = 1;
    int kind = op.kind;
    switch (op.kind) {
    case OP_INIT:
        units = im.K;
        group = 32;
        break;
    case OP_MPHASE:
    case OP_PHASE:
        if (op.level == 0) {  // warp tiles
            units = pixel_tiles(im, op.phase, cphase);
            group = 32;
        } else if (wide && op.kind == OP_PHASE && level_group(im, op.level) == 32) {  // warp blocks in tiles
            kind = OP_BTILE;
            units = level_tiles(im, op.level, op.phase, cphase);
            group = 32;
        } else {
            int cols, rows;
            lattice(im.nbx[op.level], im.nby[op.level], op.phase, cphase, &cols, &rows);
            units = (int64_t)cols * rows;
            group = level_group(im, op.level);
            if (group == 1 && small_tiles_2d(im, op.level))
                threads = (int64_t)((cols + kSmallTileX - 1) / kSmallTileX) * ((rows + kSmallTileY - 1) / kSmallTileY) * 32;
        }
        break;
    case OP_MINIT:  // a thread per pixel
        units = (int64_t)im.W * im.H;
        break;
    case OP_DESCEND:  // a thread per kRowChunk cells of a row of the finer grid
        units = (int64_t)im.nby[op.level - 1] * ((im.nbx[op.level - 1] + kRowChunk - 1) / kRowChunk);
        break;
    default:  // OP_OUTPUT: a thread per kRowChunk pixels of a row
        units = (int64_t)im.H * ((im.W + kRowChunk - 1) / kRowChunk);
        break;
    }
    const int64_t count = threads >= 0 ? threads : (units * group + 31) / 32 * 32;
    if (count > 0) {
        StepEntry e{img, kind, op.level, op.phase, o, (int32_t)units, *vt, group, cphase};
        out[n++] = e;
        *vt += count;
    }
    return n;
}

// Which phases of a step fuse their replays (emit_entries' `fuse`).  A step
// whose fused work is below `split_below` warps (the machine's warp slots)
// is bound by its slowest unit, and a unit that replays a move and then
// judges is the slowest, so the replays of block phases go to catch-up
// entries that run beside the judges; a pixel tile shares its staged labels
// between replay and judge, so its replays move out only when the step is
// below an eighth of the machine.  A full step keeps them fused, which
// takes fewer warps.  `fused_vt` is the step's thread count with fused
// entries.
__host__ __device__ inline int fuse_step(int64_t fused_vt, int64_t split_below)
{
    return fused_vt / 32 >= split_below ? 2 : fused_vt / 32 >= split_below / 8 ? 1 : 0;
}

// The mode of a step (emit_entries' `mode`): its fusion, and kWideStep when
// the step has at least kTileRounds warp tiles per warp slot of the machine.
// A wide step runs the phases of warp-judged blocks in warp tiles: a tile
// stages its block labels once and judges only its boundary blocks, which
// cuts the per-block cost of steps with many blocks.  Blocks judged by a
// thread each keep their per-unit op: a lane per block already runs 32
// judges at once.  Its catch-ups read more decisions per lane and replay
// more moves per warp (kCatchupPerLane), which pays once the machine is
// full.  With fewer units the per-unit forms keep more warps busy and each
// warp's chain of dependent loads short.
// `fused_vt`: the step's thread count with fused per-unit entries,
// `tiled_vt`: with fused tile entries.
// `policy` (seeds_tuning.block_tiles): 0 by that rule, 1 never, 2 always.
constexpr int kTileRounds = 2;
__host__ __device__ inline int step_mode(int64_t fused_vt, int64_t tiled_vt, int64_t split_below, int policy = 0)
{
    const bool tiles = policy == 2 || (policy == 0 && tiled_vt / 32 >= kTileRounds * split_below);
    return fuse_step(fused_vt, split_below) | (tiles ? kWideStep : 0);
}

// An epoch of the serving runtime: for each resident slot, the range of its
// ops to run; the device builds the step schedule from it.
constexpr int kMaxEpochSlots = 128;
struct EpochSlot {
    int32_t slot;
    int32_t begin, end;  // ops [begin, end) of the slot's image
    int32_t catchup;     // op begin-1's moves are pending
};
struct EpochPlan {
    int32_t n;            // slots in the epoch
    int32_t nsteps;       // max over slots of end - begin (<= 1024)
    int32_t split_below;  // fuse_step's threshold in warps
    int32_t tile_policy;  // step_mode's policy (seeds_tuning.block_tiles)
    EpochSlot s[kMaxEpochSlots];
};

// launch helpers (seeds_kernels.cu)
cudaError_t launch_admit(DevImage *d_imgs, int slot, const DevImage &rec, cudaStream_t s);
cudaError_t launch_epoch_schedule(const DevImage *d_imgs, const EpochPlan &plan, StepEntry *ent, int32_t *first,
                                  int64_t *vt, cudaStream_t s);
cudaError_t launch_set_io(DevImage *d_imgs, const IoChunk &chunk, cudaStream_t s);
cudaError_t launch_persistent(const DevImage *d_imgs, const Schedule &sch, GridBarrier *bar, int32_t *err,
                              int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t persistent_max_blocks_per_sm(int threads, size_t smem, int *n);
cudaError_t prepare_persistent(size_t smem);
// The LAB conversion tables (1 KB) on the current device, copied on stream
// `s` on every call made while `s` is not being captured, so that a device
// reset (which clears the module's static arrays) is followed by a fresh
// copy; a call made during a capture relies on an earlier copy on the device.
cudaError_t upload_lab_tables(cudaStream_t s);
cudaError_t launch_recount(const DevImage *d_imgs, int img, int level, int64_t npix, cudaStream_t s);

}  // namespace seeds
