// seeds_kernels.cu -- sm_103a kernels of the SEEDS hot path.
//
// One persistent kernel runs a whole schedule (see seeds_device.cuh):
//   op_init        quantise RGB to colour bins (one warp per initial
//                  superpixel rectangle), build its histogram with
//                  warp-aggregated shared-memory atomics, write the grid
//                  labels (Sec. 5.1, Eq. 4)
//   op_block_phase_warp / op_block_phase_thread / op_pixel_tile
//                  judge every unit of one parity phase against the state
//                  at phase start (Sec. 5.2-5.3: Prop. 1 for blocks, Prop. 1 +
//                  Prop. 2 for pixels); accepted moves update the other state
//                  buffer at once (the incremental histogram update of
//                  Sec. 5.3)
//   op_catchup     replay the previous phase's moves into the buffer that
//                  phase read, so both buffers stay one step apart
//   op_descend     copy block labels to the next finer grid (coarse to fine)
//   op_means_init / op_means_tile
//                  the optional means-based pixel iterations (Sec. 6.3, 6.5)
//   op_output      int32 labels for the caller; anytime_output the partition
//                  of a launch stopped early (Sec. 5.4)
// Every step ends in a grid barrier that spins with a time limit; a barrier
// that runs out sets the error word and every block leaves the kernel.  Work
// inside a step is dealt to the CTAs in rounds and taken by their warps as
// they finish (a step that fits in one round: round-robin over the CTAs).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "seeds_device.cuh"
#include "seeds_host.h"

namespace seeds {

constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int32_t *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier without a stop decision: the arrival counter only grows
// (zeroed before the launch), so barrier number s is passed once it reaches
// (s+1) * gridDim.x: one atomic per CTA, no reset, no second word.  After the
// CTA barrier, thread 0 fences (making the CTA's writes visible at gpu scope)
// and arrives; it polls with acquire loads, and the closing CTA barrier
// orders the CTA's later loads after that acquire.  A release atomic in place
// of the fence did not make the other warps' writes visible in tests, and a
// second fence after the wait costs ~0.4 us per step for nothing the acquire
// does not already give.  Returns false when the wait ran out or another CTA
// reported an error.  A CTA with arrive == false (a failure test) waits
// without arriving, so that the wait of every CTA runs out.
__device__ bool grid_sync_count(GridBarrier *bar, int32_t *err, unsigned target, uint64_t limit_ns, bool arrive)
{
    __shared__ int s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned v = arrive ? atomicAdd(&bar->count, 1u) : 0u;
        if (!arrive || v + 1 != target) {
            const uint64_t t0 = global_ns();
            for (unsigned it = 1; (int)(ld_acquire_u32(&bar->count) - target) < 0; ++it) {
                if ((it & 31u) == 0) {
                    if (ld_relaxed_i32(err) != 0) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > limit_ns) {
                        atomicOr(err, DERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(32);
            }
        }
        s_go = ok;
    }
    __syncthreads();
    return s_go != 0;
}

constexpr unsigned kGenStop = 0x80000000u;  // generation bit: the grid stops here

// Grid-wide barrier for a persistent launch whose blocks are all resident.
// Returns 0 when the wait ran out or another block reported an error, 1 to
// go on, 2 to stop: the last block to arrive decides (its thread 0 passes
// want_stop) and publishes the decision in the generation word it bumps.  A
// CTA with arrive == false (a failure test) waits without arriving.
__device__ int grid_sync(GridBarrier *bar, int32_t *err, bool want_stop, uint64_t limit_ns, bool arrive)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_u32(&bar->gen);
        __threadfence();
        const unsigned arrived = arrive ? atomicAdd(&bar->count, 1u) + 1u : 0u;
        if (arrived == gridDim.x) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, want_stop ? kGenStop + 1u : 1u);
            if (want_stop) ok = 2;
        } else {
            const uint64_t t0 = global_ns();
            unsigned cur;
            for (unsigned it = 1; (cur = ld_acquire_u32(&bar->gen)) == g; ++it) {
                if ((it & 31u) == 0) {
                    if (ld_relaxed_i32(err) != 0) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > limit_ns) {
                        atomicOr(err, DERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(32);
            }
            if (ok && ((cur ^ g) & kGenStop)) ok = 2;
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

// Debug builds (SEEDS_DEBUG_BOUNDS): every histogram, size, bin, label and
// decision index is checked against its buffer; one outside is recorded in
// the error word (DERR_BOUNDS, reported as SEEDS_ERR_DEVICE) and replaced by
// 0, so the access stays inside the buffer.  Release builds check nothing.
#ifdef SEEDS_DEBUG_BOUNDS
__device__ __forceinline__ int64_t checked_index(const DevImage &im, int64_t i, int64_t n)
{
    if (i < 0 || i >= n) {
        atomicOr(im.err, DERR_BOUNDS);
        return 0;
    }
    return i;
}
#define SEEDS_IDX(im, i, n) checked_index((im), (int64_t)(i), (int64_t)(n))
#else
#define SEEDS_IDX(im, i, n) (i)
#endif

__device__ __forceinline__ int hidx(const DevImage &im, int k, int j)
{
    return (int)SEEDS_IDX(im, k, im.K) * im.hist_sk + (int)SEEDS_IDX(im, j, im.nbins) * im.hist_sj;
}

__device__ __forceinline__ int bin_at(const DevImage &im, int p)
{
    const int64_t q = SEEDS_IDX(im, p, (int64_t)im.W * im.H);
    return im.bins16 ? (int)((const uint16_t *)im.bins)[q] : (int)((const uint8_t *)im.bins)[q];
}

// Ring of a unit, bit r: NW, N, NE, E, SE, S, SW, W (r = 0..7).  Odd bits
// are the 4-neighbours; cyclically consecutive bits are 4-adjacent cells, so
// a 4-connected set of ring cells is a cyclic run of set bits.  Leaving is
// allowed when some 4-neighbour is set and exactly one run holds
// 4-neighbours (runs made of a lone corner do not count).
__device__ __forceinline__ bool ring_allows_leaving(unsigned m)
{
    if ((m & 0xAAu) == 0) return false;
    if (m == 0xFFu) return true;
    const unsigned prev = ((m << 1) | (m >> 7)) & 0xFFu;  // bit r = bit r-1 of m
    const unsigned next = ((m >> 1) | (m << 7)) & 0xFFu;  // bit r = bit r+1 of m
    const unsigned starts = m & ~prev;
    const unsigned lone_corners = m & ~prev & ~next & 0x55u;
    return __popc(starts) - __popc(lone_corners) == 1;
}

// label of grid cell (x,y) or kNoLabel outside
__device__ __forceinline__ int cell(const uint16_t *lab, int nx, int ny, int x, int y)
{
    return (x < 0 || y < 0 || x >= nx || y >= ny) ? (int)kNoLabel : (int)lab[y * nx + x];
}

// Boundary test and ring validity of a unit over a fetch function for its
// 8-ring (cells outside the grid read kNoLabel): true when some 4-neighbour
// has another label and leaving label k keeps k 4-connected (R5, R7).
template <class Fetch>
__device__ __forceinline__ bool may_leave(Fetch at, int k)
{
    const int lf = at(-1, 0), rt = at(1, 0);
    const int up = at(0, -1), dn = at(0, 1);
    const bool boundary = (lf != k && lf != kNoLabel) || (rt != k && rt != kNoLabel) ||
                          (up != k && up != kNoLabel) || (dn != k && dn != kNoLabel);
    if (!boundary) return false;
    unsigned m = 0;
    m |= (at(-1, -1) == k) << 0;
    m |= (up == k) << 1;
    m |= (at(1, -1) == k) << 2;
    m |= (rt == k) << 3;
    m |= (at(1, 1) == k) << 4;
    m |= (dn == k) << 5;
    m |= (at(-1, 1) == k) << 6;
    m |= (lf == k) << 7;
    return ring_allows_leaving(m);
}

// The distinct labels other than k among the four neighbours, in fixed
// slots in ascending order; a slot holds kNoLabel when its label is k, a
// repeat or no label, so later loops index them with constants.  Returns
// how many there are.
__device__ __forceinline__ int sorted_candidates(int a, int b, int c, int d, int k, int cand[4])
{
    int t;
#define SEEDS_CSWAP(p, q) \
    if (p > q) {          \
        t = p;            \
        p = q;            \
        q = t;            \
    }
    SEEDS_CSWAP(a, b) SEEDS_CSWAP(c, d) SEEDS_CSWAP(a, c) SEEDS_CSWAP(b, d) SEEDS_CSWAP(b, c)
#undef SEEDS_CSWAP
    cand[0] = (a != k) ? a : (int)kNoLabel;
    cand[1] = (b != k && b != a) ? b : (int)kNoLabel;
    cand[2] = (c != k && c != b) ? c : (int)kNoLabel;
    cand[3] = (d != k && d != c) ? d : (int)kNoLabel;
    return (cand[0] != kNoLabel) + (cand[1] != kNoLabel) + (cand[2] != kNoLabel) + (cand[3] != kNoLabel);
}

// Shared unit logic: boundary test, ring validity, sorted distinct
// candidates.  Returns the candidate count (0 = no move possible).
template <class Fetch>
__device__ __forceinline__ int candidates_from(Fetch at, int k, int cand[4])
{
    if (!may_leave(at, k)) return 0;
    return sorted_candidates(at(-1, 0), at(1, 0), at(0, -1), at(0, 1), k, cand);
}

__device__ __forceinline__ int unit_candidates(const uint16_t *lab, int nx, int ny, int x, int y, int k, int cand[4])
{
    return candidates_from([&](int dx, int dy) { return cell(lab, nx, ny, x + dx, y + dy); }, k, cand);
}

// position of unit u of a parity phase on a grid nx wide
__device__ __forceinline__ void unit_pos(int u, int phase, int nx, int *x, int *y)
{
    const int px = phase & 1, py = phase >> 1;
    const int ncols = (nx - px + 1) >> 1;
    const int uy = u / ncols, ux = u - uy * ncols;
    *x = 2 * ux + px;
    *y = 2 * uy + py;
}

__device__ __forceinline__ void move_counts(const DevImage &im, int buf, int k, int n, int j, int cnt)
{
    atomicSub(&im.hist[buf][hidx(im, k, j)], cnt);
    atomicAdd(&im.hist[buf][hidx(im, n, j)], cnt);
}

__device__ __forceinline__ void move_size(const DevImage &im, int buf, int k, int n, int cnt)
{
    atomicSub(&im.size[buf][SEEDS_IDX(im, k, im.K)], cnt);
    atomicAdd(&im.size[buf][SEEDS_IDX(im, n, im.K)], cnt);
}

// The compactness prior (Sec. 6.4) keeps every superpixel's coordinate sums
// (msum entries 3 and 4) exact through every move.  Sum of x over [x0, x1):
__device__ __forceinline__ unsigned long long range_sum(int x0, int x1)
{
    const long long a = x1 - x0;
    return (unsigned long long)(a * x0 + a * (a - 1) / 2);
}

// move the coordinate sums of the rectangle [x0,x1) x [y0,y1) from k to n in
// buffer `buf`
__device__ __forceinline__ void move_xy(const DevImage &im, int buf, int k, int n, int x0, int x1, int y0, int y1)
{
    const unsigned long long sx = range_sum(x0, x1) * (unsigned long long)(y1 - y0);
    const unsigned long long sy = range_sum(y0, y1) * (unsigned long long)(x1 - x0);
    unsigned long long *mk = im.msum[buf] + (int64_t)SEEDS_IDX(im, k, im.K) * 5;
    unsigned long long *mn = im.msum[buf] + (int64_t)SEEDS_IDX(im, n, im.K) * 5;
    atomicAdd(mk + 3, 0ull - sx);
    atomicAdd(mn + 3, sx);
    atomicAdd(mk + 4, 0ull - sy);
    atomicAdd(mn + 4, sy);
}

constexpr int kHistRound = 4;  // bins loaded per lane before any is used

// Sparse colour histogram of the block [x0,x1) x [y0,y1) in the warp's
// shared scratch: counts in hsh[j], distinct bins listed in lst[0..nd).
// Whole warp; returns nd.  A lane loads kHistRound bins before it uses any.
__device__ int block_sparse_hist(const DevImage &im, int x0, int x1, int y0, int y1, int lane, int32_t *wsh,
                                 int max_nbins)
{
    int32_t *ndist = wsh;
    int32_t *hsh = wsh + kScratchHeader;
    // the list lives past the largest histogram of the context, so that it
    // never overlaps histogram entries another image's blocks rely on being 0
    uint16_t *lst = (uint16_t *)(hsh + max_nbins);
    const int bw = x1 - x0, m = bw * (y1 - y0);
    for (int base = 0; base < m; base += 32 * kHistRound) {
        int j[kHistRound];
#pragma unroll
        for (int q = 0; q < kHistRound; ++q) {
            const int t = base + 32 * q + lane;
            j[q] = -1;
            if (t < m) {
                const int dy = t / bw;
                j[q] = bin_at(im, (y0 + dy) * im.W + x0 + (t - dy * bw));
            }
        }
#pragma unroll
        for (int q = 0; q < kHistRound; ++q) {
            if (base + 32 * q >= m) break;  // m is the warp's: the rest of the round is empty
            const unsigned peers = __match_any_sync(0xffffffffu, j[q]);
            if (j[q] >= 0 && lane == __ffs(peers) - 1) {
                const int old = atomicAdd(&hsh[j[q]], __popc(peers));
                if (old == 0) lst[atomicAdd(ndist, 1)] = (uint16_t)j[q];
            }
        }
    }
    __syncwarp();
    return *(volatile int32_t *)ndist;
}

// after block_sparse_hist: apply (if k >= 0) the block's counts as a move
// k -> n to buffer `buf`, and clear the scratch for the next use
__device__ void block_sparse_apply_clear(const DevImage &im, int buf, int k, int n, int nd, int lane, int32_t *wsh,
                                         int max_nbins)
{
    int32_t *hsh = wsh + kScratchHeader;
    const uint16_t *lst = (const uint16_t *)(hsh + max_nbins);
    for (int t = lane; t < nd; t += 32) {
        const int j = lst[t];
        if (k >= 0) move_counts(im, buf, k, n, j, hsh[j]);
        hsh[j] = 0;
    }
    __syncwarp();
    if (lane == 0) wsh[0] = 0;
    __syncwarp();
}

// ---------------------------------------------------------------------------
// CIE L*a*b* colour codes (Sec. 6.2), exact integer fixed point
// ---------------------------------------------------------------------------

// sRGB byte -> linear light * 2^24; sRGB->XYZ matrix rows over the D65 white
// (the row sums) * 2^20.  Built on the host from the published definitions.
__device__ int32_t g_lab_lin[256];
__device__ int32_t g_lab_m[9];

// floor(cbrt(n)) for 0 <= n < 2^61: a single-precision estimate is within
// one of the answer; integer cubes settle it exactly
__device__ __forceinline__ int64_t icbrt_floor(int64_t n)
{
    int64_t r = (int64_t)cbrtf((float)n);
    while (r > 0 && r * r * r > n) --r;
    while ((r + 1) * (r + 1) * (r + 1) <= n) ++r;
    return r;
}

// floor(f(t) * 2^20), t = T / 2^44: t^(1/3) above (6/29)^3 = 216/24389, the
// line (24389 t + 432) / 3132 below
__device__ __forceinline__ int64_t lab_f_q20(int64_t T)
{
    if (T * 24389 > ((int64_t)216 << 44)) return icbrt_floor(T << 16);
    return (24389 * T + ((int64_t)432 << 44)) / ((int64_t)3132 << 24);
}

__device__ __forceinline__ int clamp_byte(int64_t v) { return v < 0 ? 0 : v > 255 ? 255 : (int)v; }

// 8-bit L*a*b* code of one pixel: L* * 255/100, a* + 128, b* + 128, each
// rounded half up (the numerators are >= 0 for every sRGB byte triple)
__device__ __forceinline__ void lab8(int r, int g, int b, int &c0, int &c1, int &c2)
{
    const int64_t lr = __ldg(&g_lab_lin[r]), lg = __ldg(&g_lab_lin[g]), lb = __ldg(&g_lab_lin[b]);
    int64_t f[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        f[i] = lab_f_q20(__ldg(&g_lab_m[3 * i]) * lr + __ldg(&g_lab_m[3 * i + 1]) * lg + __ldg(&g_lab_m[3 * i + 2]) * lb);
    const int64_t Lq = 116 * f[1] - ((int64_t)16 << 20);
    c0 = clamp_byte((Lq * 255 + ((int64_t)50 << 20)) / ((int64_t)100 << 20));
    c1 = clamp_byte((500 * (f[0] - f[1]) + ((int64_t)128 << 20) + (1 << 19)) >> 20);
    c2 = clamp_byte((200 * (f[1] - f[2]) + ((int64_t)128 << 20) + (1 << 19)) >> 20);
}

// ---------------------------------------------------------------------------
// op_init: one warp per initial superpixel rectangle
// ---------------------------------------------------------------------------

// Edge snapping (Sec. 6.4): the edge mask of the rectangle [x0,x1) x
// [y0,y1), a lane per column.  Bit 0 of a pixel is set when it and its right
// neighbour, bit 1 when it and the pixel below, have colour codes at least
// the threshold apart (L1 over the 3 codes).
__device__ __noinline__ void edge_mask_rect(const DevImage &im, int x0, int x1, int y0, int y1, int lane)
{
    for (int y = y0; y < y1; ++y)
        for (int x = x0 + lane; x < x1; x += 32) {
            int c[3][3];
            for (int d = 0; d < 3; ++d) {  // the pixel, its right neighbour, the pixel below
                const int qx = min(x + (d == 1), im.W - 1), qy = min(y + (d == 2), im.H - 1);
                const uint8_t *px = im.rgb + (int64_t)qy * im.stride + 3 * (int64_t)qx;
                c[d][0] = px[0];
                c[d][1] = px[1];
                c[d][2] = px[2];
                if (im.color) lab8(c[d][0], c[d][1], c[d][2], c[d][0], c[d][1], c[d][2]);
            }
            uint8_t m = 0;
            for (int d = 1; d < 3; ++d) {
                const bool inside = d == 1 ? x + 1 < im.W : y + 1 < im.H;
                const int l1 = abs(c[d][0] - c[0][0]) + abs(c[d][1] - c[0][1]) + abs(c[d][2] - c[0][2]);
                if (inside && l1 >= im.edge_tau) m |= (uint8_t)(1u << (d - 1));
            }
            im.edges[SEEDS_IDX(im, (int64_t)y * im.W + x, (int64_t)im.W * im.H)] = m;
        }
}

__device__ void op_init(const DevImage &im, int k, int lane, int32_t *wsh)
{
    if (k >= im.K) return;
    int32_t *hsh = wsh + kScratchHeader;
    const int sx = k % im.gx, sy = k / im.gx;
    const int x0 = (int)((int64_t)sx * im.W / im.gx), x1 = (int)((int64_t)(sx + 1) * im.W / im.gx);
    const int y0 = (int)((int64_t)sy * im.H / im.gy), y1 = (int)((int64_t)(sy + 1) * im.H / im.gy);
    const int w = x1 - x0, area = w * (y1 - y0);
    const int B = im.B;
    // The rectangle's pixels in row-major order, 256 per round: lane l takes
    // pixels l, l + 32, ..., l + 224 of the round, so every lane has work in
    // every round but the last whatever the rectangle's width.  A position
    // (x, y) steps 32 pixels on by (32 % w, 32 / w) and at most one wrap.
    const int step_y = 32 / w, step_x = 32 - step_y * w;
    int x = lane % w, y = lane / w;  // relative to (x0, y0)
    for (int i0 = 0; i0 < area; i0 += 256) {
        int j[8];
        const int rx = x, ry = y;  // the round's first position, walked again for the stores
        // the round's 24 byte loads first, then the arithmetic on them
        uint32_t rgb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            rgb[q] = 0xFFFFFFFFu;
            if (y0 + y < y1) {
                const uint8_t *px = im.rgb + (int64_t)(y0 + y) * im.stride + 3 * (int64_t)(x0 + x);
                rgb[q] = (uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16);
            }
            x += step_x;
            y += step_y;
            if (x >= w) {
                x -= w;
                ++y;
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            j[q] = -1;
            if (rgb[q] != 0xFFFFFFFFu) {
                int r = rgb[q] & 255, g = (rgb[q] >> 8) & 255, b = (rgb[q] >> 16) & 255;
                if (im.color) lab8(r, g, b, r, g, b);
                j[q] = ((r * B) >> 8) * B * B + ((g * B) >> 8) * B + ((b * B) >> 8);
            }
        }
        int cx = rx, cy = ry;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (j[q] >= 0) {  // a pixel of the rectangle
                const int p = (y0 + cy) * im.W + x0 + cx;
                if (im.bins16)
                    ((uint16_t *)im.bins)[p] = (uint16_t)j[q];
                else
                    ((uint8_t *)im.bins)[p] = (uint8_t)j[q];
                if (im.L == 0) im.lab[0][0][p] = im.lab[0][1][p] = (uint16_t)k;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, j[q]);
            if (j[q] >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hsh[j[q]], __popc(peers));
            cx += step_x;
            cy += step_y;
            if (cx >= w) {
                cx -= w;
                ++cy;
            }
        }
    }
    if (im.edges) edge_mask_rect(im, x0, x1, y0, y1, lane);
    __syncwarp();
    for (int j = lane; j < im.nbins; j += 32) {
        const int v = hsh[j];
        im.hist[0][hidx(im, k, j)] = v;
        im.hist[1][hidx(im, k, j)] = v;
        hsh[j] = 0;
    }
    __syncwarp();
    if (lane == 0) im.size[0][k] = im.size[1][k] = area;
    if (im.msum[0] && lane < 10) {  // colour sums zero; with the prior, the rectangle's coordinate sums
        const int q = lane % 5;
        unsigned long long v = 0;
        if (im.prior && q == 3) v = range_sum(x0, x1) * (unsigned long long)(y1 - y0);
        if (im.prior && q == 4) v = range_sum(y0, y1) * (unsigned long long)(x1 - x0);
        im.msum[lane / 5][(int64_t)k * 5 + q] = v;
    }
    {  // every decision "no move": the judges write moves only, and replays reset what they read
        const int64_t chunk = (im.units_cap + im.K - 1) / im.K;
        const int64_t e0 = (int64_t)k * chunk, e1 = min(e0 + chunk, (int64_t)im.units_cap);
        for (int64_t e = e0 + lane; e < e1; e += 32) im.dec[0][e] = im.dec[1][e] = kNoMove;
    }
    if (im.L >= 1 && lane < 4) {
        const int L = im.L;
        const int bx = 2 * sx + (lane & 1), by = 2 * sy + (lane >> 1);
        im.lab[L][0][by * im.nbx[L] + bx] = im.lab[L][1][by * im.nbx[L] + bx] = (uint16_t)k;
    }
}

// ---------------------------------------------------------------------------
// means-based pixel iterations (SPM, Sec. 6.3; the last pixel iterations,
// Sec. 6.5): per superpixel sums of the colour codes and coordinates
// ---------------------------------------------------------------------------

// colour code of pixel (x, y): its RGB bytes or their 8-bit L*a*b* code
__device__ __noinline__ void pixel_code(const DevImage &im, int x, int y, int &c0, int &c1, int &c2)
{
    const uint8_t *px = im.rgb + (int64_t)y * im.stride + 3 * (int64_t)x;
    c0 = px[0];
    c1 = px[1];
    c2 = px[2];
    if (im.color) lab8(c0, c1, c2, c0, c1, c2);
}

// move pixel (x, y) from k to n in the sums of buffer `buf`
__device__ __noinline__ void move_sums(const DevImage &im, int buf, int k, int n, int x, int y)
{
    int c0, c1, c2;
    pixel_code(im, x, y, c0, c1, c2);
    const unsigned long long v[5] = {(unsigned long long)c0, (unsigned long long)c1, (unsigned long long)c2,
                                     (unsigned long long)x, (unsigned long long)y};
    unsigned long long *mk = im.msum[buf] + (int64_t)k * 5, *mn = im.msum[buf] + (int64_t)n * 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        atomicAdd(mk + q, 0ull - v[q]);
        atomicAdd(mn + q, v[q]);
    }
}

// OP_MINIT: the sums from the labels of buffer o&1, into both buffers (zeroed
// by the init op; with the compactness prior the coordinate sums are already
// kept, so only the colour sums are added).  A thread per pixel; the warp adds up each label's lanes
// and one lane per label adds them to memory.  The whole warp calls this.
__device__ __noinline__ void op_means_init(const DevImage &im, int o, int64_t units, int64_t t, int lane)
{
    int k = -1;
    unsigned v[5] = {0, 0, 0, 0, 0};
    if (t < units) {
        const int y = (int)(t / im.W), x = (int)(t - (int64_t)y * im.W);
        k = im.lab[0][o & 1][t];
        int c0, c1, c2;
        pixel_code(im, x, y, c0, c1, c2);
        v[0] = c0;
        v[1] = c1;
        v[2] = c2;
        v[3] = x;
        v[4] = y;
    }
    unsigned todo = 0xffffffffu;  // the same on every lane
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int kl = __shfl_sync(0xffffffffu, k, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, k == kl);
        unsigned s[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] = __reduce_add_sync(0xffffffffu, k == kl ? v[q] : 0u);
        if (lane == leader && kl >= 0)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (q >= 3 && im.prior) break;
                atomicAdd(&im.msum[0][(int64_t)kl * 5 + q], (unsigned long long)s[q]);
                atomicAdd(&im.msum[1][(int64_t)kl * 5 + q], (unsigned long long)s[q]);
            }
        todo &= ~grp;
    }
}

// SLIC's squared distance of a pixel (codes c, position x, y) to the mean of
// superpixel `label` in buffer b: colour, plus (m/S)^2 times the squared
// distance to the centroid, in IEEE single precision, one rounding per
// operation in this order (no fused multiply-add); a mean is its sum times
// 1/|A|
__device__ __forceinline__ float means_distance(const DevImage &im, int b, int label, const int c[3], int x, int y)
{
    const unsigned long long *m = im.msum[b] + (int64_t)label * 5;
    const float r = __fdiv_rn(1.0f, __int2float_rn(im.size[b][label]));
    float dc = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float t = __fsub_rn(__int2float_rn(c[q]), __fmul_rn(__ll2float_rn((long long)m[q]), r));
        dc = __fadd_rn(dc, __fmul_rn(t, t));
    }
    const float gx = __fsub_rn(__int2float_rn(x), __fmul_rn(__ll2float_rn((long long)m[3]), r));
    const float gy = __fsub_rn(__int2float_rn(y), __fmul_rn(__ll2float_rn((long long)m[4]), r));
    const float ds = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
    return __fadd_rn(dc, __fmul_rn(im.means_w, ds));
}

// The means rule for boundary pixel p = (x, y) of label k that may leave:
// the candidate (ascending, empty slots kNoLabel) whose mean is nearest,
// ties to the smallest label, if strictly nearer than k's mean (p
// included).  A move is applied to buffer nb at once.
__device__ __noinline__ uint32_t means_pixel(const DevImage &im, int b, int nb, int x, int y, int k, int j,
                                             const int cand[4])
{
    int c[3];
    pixel_code(im, x, y, c[0], c[1], c[2]);
    int best = kNoLabel;
    float db = 0.0f;
    for (int q = 0; q < 4; ++q) {
        const int n = cand[q];
        if (n == kNoLabel) continue;
        const float d = means_distance(im, b, n, c, x, y);
        if (best == kNoLabel || d < db) {
            best = n;
            db = d;
        }
    }
    if (!(db < means_distance(im, b, k, c, x, y))) return kNoMove;
    im.lab[0][nb][SEEDS_IDX(im, y * im.W + x, (int64_t)im.W * im.H)] = (uint16_t)SEEDS_IDX(im, best, im.K);
    move_counts(im, nb, k, best, j, 1);
    move_size(im, nb, k, best, 1);
    move_sums(im, nb, k, best, x, y);
    return ((uint32_t)k << 16) | (uint32_t)best;
}

// ---------------------------------------------------------------------------
// the compactness prior (Sec. 6.4) in the histogram pixel phases
// ---------------------------------------------------------------------------

// The pixel score of one option: D*a/s + gamma*G - compact_w*d^2, d^2 the
// squared distance of (x, y) to the centre of gravity of `label` in buffer b
// (coordinate sums over sc pixels), in IEEE single precision with one
// rounding per operation in this order (no fused multiply-add).
__device__ __forceinline__ float compact_score(const DevImage &im, int b, int label, int x, int y, int32_t a,
                                               int32_t s, int32_t sc, int G)
{
    const unsigned long long *m = im.msum[b] + (int64_t)label * 5;
    const float r = __fdiv_rn(1.0f, __int2float_rn(sc));
    const float gx = __fsub_rn(__int2float_rn(x), __fmul_rn(__ll2float_rn((long long)m[3]), r));
    const float gy = __fsub_rn(__int2float_rn(y), __fmul_rn(__ll2float_rn((long long)m[4]), r));
    const float d2 = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
    const float col = __fdiv_rn(__int2float_rn(a), __int2float_rn(s));
    const float t1 = __fmul_rn(81.0f, col);
    const float t2 = __fmul_rn(im.gamma_f, __int2float_rn(G));
    const float t3 = __fmul_rn(im.compact_w, d2);
    return __fsub_rn(__fadd_rn(t1, t2), t3);
}

// The best candidate (ascending, a later one only if strictly higher: ties to
// the smallest label) if its score is strictly above staying, else kNoLabel.
// A candidate scores its colour count A_n[j] and size |A_n| with
// G_n + |K_p|; staying scores A_k without the pixel (A_k[j] - 1, |A_k| - 1)
// with G_k, its centre taken with the pixel in it.  The candidate labels
// come packed two to a word (kNoLabel in empty slots), their G values a
// byte each (at most 81); the counts are looked up here.
__device__ __noinline__ int compact_pick(const DevImage &im, int b, int x, int y, int k, int j, uint32_t c01,
                                         uint32_t c23, uint32_t gpack, int Kp, int Gk)
{
    const int32_t *hist = im.hist[b], *size = im.size[b];
    int best = kNoLabel;
    float fb = 0.0f;
    for (int c = 0; c < 4; ++c) {
        const int n = (int)(((c < 2 ? c01 : c23) >> (16 * (c & 1))) & 0xFFFFu);
        if (n == kNoLabel) continue;
        const int32_t a = hist[hidx(im, n, j)], sz = size[SEEDS_IDX(im, n, im.K)];
        const float f = compact_score(im, b, n, x, y, a, sz, sz, (int)((gpack >> (8 * c)) & 0xFFu) + Kp);
        if (best == kNoLabel || f > fb) {
            best = n;
            fb = f;
        }
    }
    const int32_t a_k = hist[hidx(im, k, j)], s_k = size[SEEDS_IDX(im, k, im.K)];
    const float fk = compact_score(im, b, k, x, y, a_k - 1, s_k - 1, s_k, Gk);
    return fb > fk ? best : (int)kNoLabel;
}

// ---------------------------------------------------------------------------
// pixel phase: warp tiles
// ---------------------------------------------------------------------------

// Edge snapping (Sec. 6.4): a unit at pixel p whose 4-neighbours (labels
// lf, rt, up, dn of the phase-start state, kNoLabel outside the image) hold
// another label across an edge of the image does not move.
__device__ __noinline__ bool edge_frozen(const DevImage &im, int p, int k, int lf, int rt, int up, int dn)
{
    const uint8_t *e = im.edges;
    return (lf != k && lf != kNoLabel && (e[p - 1] & 1)) || (rt != k && rt != kNoLabel && (e[p] & 1)) ||
           (up != k && up != kNoLabel && (e[p - im.W] & 2)) || (dn != k && dn != kNoLabel && (e[p] & 2));
}

// The labels of a warp tile plus a 2-cell halo, from a label grid nx x ny
// (kNoLabel outside), in TH rows of kTileW cells: lane l loads columns l,
// l+32 (packed in one register) and, for l < 4, l+64 of every row.  The
// loads (tile_load) are all issued before the first shared-memory store
// (tile_store, after a __syncwarp): a warp issues in order, and a store
// waits for its load, so interleaving them would serialise one L2 round trip
// per store.
template <int TH>
struct TileRegs {
    uint32_t v01[TH];
    uint16_t v2[TH];
};

template <int TH>
__device__ __forceinline__ void tile_load(TileRegs<TH> &t, const uint16_t *lab, int nx, int ny, int X0, int Y0,
                                          int lane)
{
    static_assert(kTileW > 64 && kTileW <= 96, "three columns per lane");
#pragma unroll
    for (int r = 0; r < TH; ++r) {
        const int yy = Y0 + r;
        const bool rowin = yy >= 0 && yy < ny;
        const uint16_t *row = lab + (int64_t)yy * nx;
        const int x0 = X0 + lane, x1 = x0 + 32, x2 = x0 + 64;
        const uint32_t a = (rowin && x0 >= 0 && x0 < nx) ? row[x0] : kNoLabel;
        const uint32_t c = (rowin && x1 >= 0 && x1 < nx) ? row[x1] : kNoLabel;
        t.v01[r] = a | (c << 16);
        t.v2[r] = (lane + 64 < kTileW && rowin && x2 >= 0 && x2 < nx) ? row[x2] : kNoLabel;
    }
}

template <int TH>
__device__ __forceinline__ void tile_store(const TileRegs<TH> &t, uint16_t *tsh, int lane)
{
#pragma unroll
    for (int r = 0; r < TH; ++r) {
        tsh[r * kTileW + lane] = (uint16_t)(t.v01[r] & 0xFFFFu);
        tsh[r * kTileW + lane + 32] = (uint16_t)(t.v01[r] >> 16);
        if (lane + 64 < kTileW) tsh[r * kTileW + lane + 64] = t.v2[r];
    }
}

// Replay one move k -> n of pixel p into buffer `buf`.
__device__ __forceinline__ void replay_pixel(const DevImage &im, int buf, int p, uint32_t d)
{
    const int k = (int)(d >> 16), n = (int)(d & 0xFFFFu);
    im.lab[0][buf][p] = (uint16_t)n;
    move_counts(im, buf, k, n, bin_at(im, p), 1);
    move_size(im, buf, k, n, 1);
}

// A histogram pixel phase's decision: the pixel's label k, the direction of
// the 4-neighbour whose label it takes (0 left, 1 right, 2 up, 3 down) and
// its bin j (k < 2^16, j < 2^12: below kNoMove).  A replay then needs no
// load of the bin, and reads the new label from that neighbour, which no op
// between the judge and the replay relabels: the neighbour has the other
// parity, and the buffer the next op reads holds it as the judge saw it.
__device__ __forceinline__ uint32_t pixel_dec(int k, int dir, int j)
{
    return ((uint32_t)k << 14) | ((uint32_t)dir << 12) | (uint32_t)j;
}
// the direction of a 4-neighbour of the staged cell T whose label is n
__device__ __forceinline__ int pixel_dir(const uint16_t *T, int n)
{
    return T[-1] == n ? 0 : T[1] == n ? 1 : T[-kTileW] == n ? 2 : 3;
}
// replay the decided move d of pixel (x, y) into buffer `buf`, the new label n
__device__ __forceinline__ void replay_pixel_dec(const DevImage &im, int buf, int x, int y, uint32_t d, int n)
{
    const int k = (int)(d >> 14), j = (int)(d & 0xFFFu);
    im.lab[0][buf][y * im.W + x] = (uint16_t)n;
    move_counts(im, buf, k, n, j, 1);
    move_size(im, buf, k, n, 1);
    if (im.prior) move_xy(im, buf, k, n, x, x + 1, y, y + 1);
}

// One warp-tile of a pixel phase: units (ux, uy) with ux in a 32-wide column
// range (one per lane) and uy in a UY-row range.  The warp first
// replays the moves of the previous phase (cphase >= 0) for the same unit
// range, then judges its own units.  The labels of the tile and a 2-pixel
// halo are staged in shared memory (kNoLabel outside the image) with
// independent coalesced loads, with the units' colour bins; a cheap pass
// finds the units that sit on a boundary and may leave, and the warp judges
// only those, compacted so that every lane works.
//
// MEANS: a means-based phase (OP_MPHASE), whose moves also carry the
// superpixel sums and whose units are judged by means_pixel.
template <bool MEANS, int UY>
__device__ void op_pixel_tile(const DevImage &im, int o, int phase, int cphase, int tiles, int tile, int lane,
                              uint16_t *tsh)
{
    if (tile >= tiles) return;
    const int b = o & 1, nb = b ^ 1;
    const int W = im.W, H = im.H;
    const int px = phase & 1, py = phase >> 1;
    const int ncols = (W - px + 1) >> 1, nrows = (H - py + 1) >> 1;
    int mcols, mrows;
    lattice(W, H, phase, cphase, &mcols, &mrows);
    const int tiles_x = (mcols + kTileUX - 1) / kTileUX;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int ux = tx * kTileUX + lane, uy0 = ty * UY;

    // the previous phase's decisions for the same units (loads issued first)
    uint32_t cd[UY];
    int ccols = 0, crows = 0, cpx = 0, cpy = 0;
    if (cphase >= 0) {
        cpx = cphase & 1;
        cpy = cphase >> 1;
        ccols = (W - cpx + 1) >> 1;
        crows = (H - cpy + 1) >> 1;
    }
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        const int uy = uy0 + r;
        cd[r] = (ux < ccols && uy < crows) ? im.dec[nb][SEEDS_IDX(im, uy * ccols + ux, im.units_cap)] : kNoMove;
    }

    // stage the labels of buffer b (and, in a means phase, the units' bins).
    // Every load is issued before the first shared-memory store: a warp
    // issues in order, and a store waits for its load, so interleaving them
    // would serialise one L2 round trip per store.  Lane l loads columns l,
    // l+32 (packed in one register) and, for l < 4, l+64 of each row.  A
    // histogram phase loads a unit's bin only when it judges the unit: the
    // boundary units are a tenth of the tile at 4K, and loading every
    // unit's bin read half of the bin map each phase, most of it unused
    // (4K batch: pixel phase 697 -> 651 us per step).
    constexpr int TH = tile_h(UY);
    TileRegs<TH> stage;
    tile_load<TH>(stage, im.lab[0][b], W, H, 2 * tx * kTileUX + px - 2, 2 * uy0 + py - 2, lane);
    uint16_t jv[UY];
    if constexpr (MEANS) {
#pragma unroll
        for (int r = 0; r < UY; ++r) {
            const int uy = uy0 + r;
            jv[r] = (ux < ncols && uy < nrows) ? bin_at(im, (2 * uy + py) * W + 2 * ux + px) : 0;
        }
    }
    __syncwarp();  // keeps the loads above the stores
    uint16_t *jsh = tsh + kTileW * TH;
    uint8_t *lst = (uint8_t *)(jsh + UY * kTileUX);
    tile_store<TH>(stage, tsh, lane);
    if constexpr (MEANS) {
#pragma unroll
        for (int r = 0; r < UY; ++r) jsh[r * 32 + lane] = jv[r];
    }

    // replay the previous phase's moves into buffer nb (a histogram phase's
    // new label from the staged neighbour it names)
    __syncwarp();
#pragma unroll
    for (int r = 0; r < UY; ++r)
        if (cd[r] != kNoMove) {
            const int cx = 2 * ux + cpx, cy = 2 * (uy0 + r) + cpy;
            if constexpr (MEANS) {
                replay_pixel(im, nb, cy * W + cx, cd[r]);
                move_sums(im, nb, (int)(cd[r] >> 16), (int)(cd[r] & 0xFFFFu), cx, cy);
            } else {
                const uint16_t *C = tsh + (2 * r + cpy - py + 2) * kTileW + (2 * lane + cpx - px + 2);
                const int dir = (int)(cd[r] >> 12) & 3;
                const int n = dir == 0 ? C[-1] : dir == 1 ? C[1] : dir == 2 ? C[-kTileW] : C[kTileW];
                replay_pixel_dec(im, nb, cx, cy, cd[r], n);
            }
            im.dec[nb][SEEDS_IDX(im, (uy0 + r) * ccols + ux, im.units_cap)] = kNoMove;
        }
    __syncwarp();

    // pass 1: boundary units that may leave; the others decide "stay" here
    unsigned mine = 0;
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        const int uy = uy0 + r;
        if (ux < ncols && uy < nrows) {
            const uint16_t *T = tsh + (2 * r + 2) * kTileW + (2 * lane + 2);
            if (may_leave([&](int dx, int dy) { return (int)T[dy * kTileW + dx]; }, (int)T[0]))
                mine |= 1u << r;
        }
    }
    int nbd = 0;
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        const unsigned bal = __ballot_sync(0xffffffffu, (mine >> r) & 1u);
        if ((mine >> r) & 1u) lst[nbd + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(r * 32 + lane);
        nbd += __popc(bal);
    }
    __syncwarp();

    // pass 2: judge the boundary units, every lane busy (a unit frozen by
    // edge snapping stays)
    const int32_t *hist = im.hist[b], *size = im.size[b];
    const int32_t gd81 = 81 * im.gden, gn = im.gnum;  // both below 2^17; the products below widen to 64 bits
    const bool use_g = im.patch != 0 && im.gnum != 0;
    for (int i = lane; i < nbd; i += 32) {
        const int e = lst[i], r = e >> 5, l = e & 31;
        const int uxe = tx * kTileUX + l, uy = uy0 + r;
        const int x = 2 * uxe + px, y = 2 * uy + py, p = y * W + x;
        const uint16_t *T = tsh + (2 * r + 2) * kTileW + (2 * l + 2);  // the unit's cell in the tile
        const int k = T[0];
        if (im.edges && edge_frozen(im, p, k, T[-1], T[1], T[-kTileW], T[kTileW])) continue;
        int cand[4];
        // pass 1 found that it may leave
        const int nc = sorted_candidates(T[-1], T[1], T[-kTileW], T[kTileW], k, cand);
        const int j = MEANS ? (int)jsh[r * 32 + l] : bin_at(im, p);
        if constexpr (MEANS) {
            const uint32_t dm = means_pixel(im, b, nb, x, y, k, j, cand);
            if (dm != kNoMove) im.dec[b][SEEDS_IDX(im, uy * ncols + uxe, im.units_cap)] = dm;
            continue;
        }
        // Prop. 2 sums G_x = sum_{i in K_p} b_{N_i}(x) as a weighted count
        // over the 5x5 window: w(p,q) = #{i in image: |i-p|,|i-q| <= 1}
        int Gk = 0, Gc[4] = {0, 0, 0, 0}, Kp = 0;
        if (use_g && nc == 1 && x >= 2 && y >= 2 && x + 2 < W && y + 2 < H) {
            // away from the border w(p,q) = (3-|dx|)(3-|dy|) and |K_p| = 9;
            // with one candidate (the smallest slot value: empty slots hold
            // kNoLabel) only two labels are counted
            Kp = 9;
            const int c0 = min(min(cand[0], cand[1]), min(cand[2], cand[3]));
            int G0 = 0;
#pragma unroll
            for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx) {
                    const int w = (3 - (dx < 0 ? -dx : dx)) * (3 - (dy < 0 ? -dy : dy));
                    const int lq = T[dy * kTileW + dx];
                    Gk += lq == k ? w : 0;
                    G0 += lq == c0 ? w : 0;
                }
#pragma unroll
            for (int c = 0; c < 4; ++c) Gc[c] = G0;  // read only for the slot holding c0
        } else if (use_g) {
            int wx[5], wy[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                const int qx = x + d - 2, qy = y + d - 2;
                const int lox = max(max(x, qx) - 1, 0), hix = min(min(x, qx) + 1, W - 1);
                const int loy = max(max(y, qy) - 1, 0), hiy = min(min(y, qy) + 1, H - 1);
                wx[d] = (qx < 0 || qx >= W) ? 0 : max(0, hix - lox + 1);
                wy[d] = (qy < 0 || qy >= H) ? 0 : max(0, hiy - loy + 1);
            }
            Kp = wx[2] * wy[2];
#pragma unroll
            for (int dy = 0; dy < 5; ++dy) {
                const uint16_t *row = T + (dy - 2) * kTileW - 2;
#pragma unroll
                for (int dx = 0; dx < 5; ++dx) {
                    const int w = wx[dx] * wy[dy];
                    const int lq = row[dx];
                    if (lq == k) Gk += w;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (lq == cand[c]) Gc[c] += w;  // empty slots only meet w = 0 cells
                }
            }
        }
        if (im.prior) {  // the compactness prior: single-precision scores
            const int best = compact_pick(im, b, x, y, k, j, (uint32_t)cand[0] | ((uint32_t)cand[1] << 16),
                                          (uint32_t)cand[2] | ((uint32_t)cand[3] << 16),
                                          (uint32_t)Gc[0] | ((uint32_t)Gc[1] << 8) | ((uint32_t)Gc[2] << 16) |
                                              ((uint32_t)Gc[3] << 24),
                                          Kp, Gk);
            uint32_t dec = kNoMove;
            if (best != kNoLabel) {
                dec = pixel_dec(k, pixel_dir(T, best), j);
                im.lab[0][nb][SEEDS_IDX(im, p, (int64_t)W * H)] = (uint16_t)SEEDS_IDX(im, best, im.K);
                move_counts(im, nb, k, best, j, 1);
                move_size(im, nb, k, best, 1);
                move_xy(im, nb, k, best, x, x + 1, y, y + 1);
                im.dec[b][SEEDS_IDX(im, uy * ncols + uxe, im.units_cap)] = dec;
            }
            continue;
        }
        // the histogram and size lookups of every candidate and of k, all
        // issued before the first is used
        int32_t ac[4], zc[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = cand[c] != kNoLabel ? cand[c] : k;
            ac[c] = hist[hidx(im, n, j)];
            zc[c] = size[SEEDS_IDX(im, n, im.K)];
        }
        const int32_t a_k = hist[hidx(im, k, j)], s_k = size[SEEDS_IDX(im, k, im.K)];
        // candidates in ascending label order; a later one wins only if
        // strictly better, so ties go to the smallest label.  Counts and
        // sizes are held in 32 bits and multiplied in 64.
        int best = kNoLabel;
        int32_t a_b = 0, s_b = 1;
        int G_b = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = cand[c];
            if (n == kNoLabel) continue;
            const int32_t a = ac[c], sz = zc[c];
            if (best == kNoLabel || gd81 * ((int64_t)a * s_b - (int64_t)a_b * sz) +
                                            gn * (int64_t)(Gc[c] - G_b) * sz * s_b > 0) {
                best = n;
                a_b = a;
                s_b = sz;
                G_b = Gc[c];
            }
        }
        const int64_t gain = gd81 * ((int64_t)a_b * (s_k - 1) - (int64_t)(a_k - 1) * s_b) +
                             gn * (int64_t)(G_b + Kp - Gk) * s_b * (s_k - 1);
        uint32_t dec = kNoMove;
        if (gain > 0) {
            dec = pixel_dec(k, pixel_dir(T, best), j);
            im.lab[0][nb][SEEDS_IDX(im, p, (int64_t)W * H)] = (uint16_t)SEEDS_IDX(im, best, im.K);
            move_counts(im, nb, k, best, j, 1);
            move_size(im, nb, k, best, 1);
            im.dec[b][SEEDS_IDX(im, uy * ncols + uxe, im.units_cap)] = dec;
        }
    }
    __syncwarp();
}

// A means-based phase's tile, out of line: the means iterations are rare, and
// the persistent kernel's other ops keep their code compact without it.
__device__ __noinline__ void op_means_tile(const DevImage &im, int o, int phase, int cphase, int tiles, int tile,
                                           int lane, uint16_t *tsh)
{
    if (im.tile_uy == 2)
        op_pixel_tile<true, 2>(im, o, phase, cphase, tiles, tile, lane, tsh);
    else
        op_pixel_tile<true, kTileUY>(im, o, phase, cphase, tiles, tile, lane, tsh);
}

// ---------------------------------------------------------------------------
// block phase, small blocks: one thread per block (at most 16 pixels)
// ---------------------------------------------------------------------------


// Move the colour counts of a small block's pixels (bins jj[0..m), SM
// bounding m) from k to n in buffer `buf`: one pair of atomics per distinct
// bin with its count, rather than one per pixel.
template <int SM>
__device__ __forceinline__ void move_block_counts(const DevImage &im, int buf, int k, int n, const int (&jj)[SM], int m)
{
#pragma unroll
    for (int t = 0; t < SM; ++t) {
        if (t >= m) break;
        bool first = true;
        int Lj = 0;
#pragma unroll
        for (int q = 0; q < SM; ++q) {
            if (q < t && jj[q] == jj[t]) first = false;
            if (q >= t && jj[q] == jj[t]) ++Lj;
        }
        if (first) move_counts(im, buf, k, n, jj[t], Lj);
    }
}

// Replay a small block's move into buffer `buf` (one thread); SM bounds its
// pixel count.  The block's bins are all loaded before the first atomic
// that needs one, so the loads share one trip to L2.
template <int SM>
__device__ void replay_small_block_t(const DevImage &im, int buf, int level, int bx, int by, uint32_t d)
{
    const int k = (int)(d >> 16), n = (int)(d & 0xFFFFu);
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    const int bw = x1 - x0, m = bw * (y1 - y0);
    int jj[SM];
    int p = y0 * im.W + x0, dx = 0;  // pixel t of the block, row-major, stepped without a division
#pragma unroll
    for (int t = 0; t < SM; ++t) {
        jj[t] = t < m ? bin_at(im, p) : -1;
        ++p;
        if (++dx == bw) {
            dx = 0;
            p += im.W - bw;
        }
    }
    move_block_counts<SM>(im, buf, k, n, jj, m);
    move_size(im, buf, k, n, m);
    if (im.prior) move_xy(im, buf, k, n, x0, x1, y0, y1);
    im.lab[level][buf][SEEDS_IDX(im, by * im.nbx[level] + bx, (int64_t)im.nbx[level] * im.nby[level])] =
        (uint16_t)SEEDS_IDX(im, n, im.K);
}

__device__ __forceinline__ void replay_small_block(const DevImage &im, int buf, int level, int bx, int by,
                                                   uint32_t d)
{
    const int ma = im.maxarea[level];
    if (ma <= 4)
        replay_small_block_t<4>(im, buf, level, bx, by, d);
    else if (ma <= 9)
        replay_small_block_t<9>(im, buf, level, bx, by, d);
    else
        replay_small_block_t<kSmallMax>(im, buf, level, bx, by, d);
}

// Judge small block (bx,by) of label k that may leave, with candidates
// cand (ascending, kNoLabel in empty slots); SM bounds its pixel count, so
// the dedupe of its bins unrolls to SM*SM compares.
template <int SM>
__device__ uint32_t judge_small_block_c(const DevImage &im, int b, int nb, int level, int bx, int by, int k,
                                        const int cand[4], int x0, int x1, int y0, int y1)
{
    const int nx = im.nbx[level];
    const int32_t *hist = im.hist[b], *size = im.size[b];
    const int bw = x1 - x0, m = bw * (y1 - y0);
    int jj[SM];
    int p = y0 * im.W + x0, dx = 0;  // pixel t of the block, row-major, stepped without a division
#pragma unroll
    for (int t = 0; t < SM; ++t) {
        jj[t] = t < m ? bin_at(im, p) : -1;
        ++p;
        if (++dx == bw) {
            dx = 0;
            p += im.W - bw;
        }
    }
    // the sums in 32 bits: every term is at most L_j * |A| and they add up
    // to at most |L| * N <= kSmallMax * N < 2^31 (the thread path is only
    // taken below that); the comparisons cross-multiply in 64 bits
    int32_t S[4] = {0, 0, 0, 0}, S_st = 0;
    int32_t sz[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sz[c] = cand[c] != kNoLabel ? size[SEEDS_IDX(im, cand[c], im.K)] : 1;
    const int32_t s_k = size[SEEDS_IDX(im, k, im.K)], s_rest = s_k - m;
    // S(A, L) = sum over the distinct bins j of L of min(A[j]*|L|, L_j*|A|)
#pragma unroll
    for (int t = 0; t < SM; ++t) {
        if (t >= m) break;
        const int j = jj[t];
        bool first = true;
        int Lj = 0;
#pragma unroll
        for (int q = 0; q < SM; ++q) {
            if (q < t && jj[q] == j) first = false;
            if (q >= t && jj[q] == j) ++Lj;
        }
        if (!first) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (cand[c] != kNoLabel) S[c] += min(hist[hidx(im, cand[c], j)] * m, Lj * sz[c]);
        S_st += min((hist[hidx(im, k, j)] - Lj) * m, Lj * s_rest);
    }
    // ascending candidates, strictly better replaces: ties to the smallest label
    int n = kNoLabel;
    int64_t Sb = 0, zb = 1;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (cand[c] != kNoLabel && (n == kNoLabel || (int64_t)S[c] * zb > Sb * sz[c])) {
            n = cand[c];
            Sb = S[c];
            zb = sz[c];
        }
    if (!(Sb * s_rest > (int64_t)S_st * zb)) return kNoMove;
    im.lab[level][nb][SEEDS_IDX(im, by * nx + bx, (int64_t)nx * im.nby[level])] = (uint16_t)SEEDS_IDX(im, n, im.K);
    move_block_counts<SM>(im, nb, k, n, jj, m);
    move_size(im, nb, k, n, m);
    if (im.prior) move_xy(im, nb, k, n, x0, x1, y0, y1);
    return ((uint32_t)k << 16) | (uint32_t)n;
}

// Judge small block (bx,by) from the label grid: its candidates, then the core.
template <int SM>
__device__ uint32_t judge_small_block(const DevImage &im, int b, int nb, int level, int bx, int by)
{
    const int nx = im.nbx[level], ny = im.nby[level];
    const uint16_t *lab = im.lab[level][b];
    // the block's extent is read with its labels: one trip to L2 fewer
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    const int k = lab[by * nx + bx];
    int cand[4];
    if (unit_candidates(lab, nx, ny, bx, by, k, cand) == 0) return kNoMove;
    return judge_small_block_c<SM>(im, b, nb, level, bx, by, k, cand, x0, x1, y0, y1);
}

// Thread t of the entry takes unit (ux,uy) of the union lattice (the t-th
// unit, or lane t%32 of the t/32-th block of kSmallTileX x kSmallTileY
// units, small_tiles_2d): replay the previous phase's move of that unit
// (cphase >= 0), then judge this phase's unit.
__device__ void op_block_phase_thread(const DevImage &im, int o, int level, int phase, int cphase, int units, int t)
{
    const int b = o & 1, nb = b ^ 1;
    const int nx = im.nbx[level], ny = im.nby[level];
    int mcols, mrows, ncols, nrows;
    lattice(nx, ny, phase, cphase, &mcols, &mrows);
    lattice(nx, ny, phase, -1, &ncols, &nrows);
    int ux, uy;
    if (small_tiles_2d(im, level)) {
        const int w = t >> 5, l = t & 31;
        const int tiles_x = (mcols + kSmallTileX - 1) / kSmallTileX;
        const int ty = w / tiles_x, tx = w - ty * tiles_x;
        ux = tx * kSmallTileX + l % kSmallTileX;
        uy = ty * kSmallTileY + l / kSmallTileX;
        if (ux >= mcols || uy >= mrows) return;
    } else {
        if (t >= units) return;
        uy = t / mcols;
        ux = t - uy * mcols;
    }
    if (cphase >= 0) {
        int ccols, crows;
        lattice(nx, ny, cphase, -1, &ccols, &crows);
        if (ux < ccols && uy < crows) {
            const uint32_t d = im.dec[nb][SEEDS_IDX(im, uy * ccols + ux, im.units_cap)];
            if (d != kNoMove) {
                replay_small_block(im, nb, level, 2 * ux + (cphase & 1), 2 * uy + (cphase >> 1), d);
                im.dec[nb][SEEDS_IDX(im, uy * ccols + ux, im.units_cap)] = kNoMove;
            }
        }
    }
    if (ux >= ncols || uy >= nrows) return;
    const int bx = 2 * ux + (phase & 1), by = 2 * uy + (phase >> 1);
    const int ma = im.maxarea[level];
    const uint32_t dec = ma <= 4   ? judge_small_block<4>(im, b, nb, level, bx, by)
                         : ma <= 9 ? judge_small_block<9>(im, b, nb, level, bx, by)
                                   : judge_small_block<kSmallMax>(im, b, nb, level, bx, by);
    if (dec != kNoMove) im.dec[b][SEEDS_IDX(im, uy * ncols + ux, im.units_cap)] = dec;
}

// ---------------------------------------------------------------------------
// block phase, large blocks: one warp per block
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t warp_sum64(int64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int32_t warp_sum(int32_t v) { return __reduce_add_sync(0xffffffffu, v); }
__device__ __forceinline__ int64_t warp_sum(int64_t v) { return warp_sum64(v); }

// The intersection sums of a block against its candidates (S) and against
// k without the block (S_st), from the warp's sparse histogram of the block:
// each lane sums its distinct bins in T, the warp adds the lanes up.
template <typename T>
__device__ __forceinline__ void warp_block_sums(const DevImage &im, int b, const int32_t *wsh, int max_nbins, int nd,
                                                int lane, int k, const int cand[4], const int32_t sz[4],
                                                int32_t s_rest, int m, int64_t S[4], int64_t &S_st)
{
    const int32_t *hist = im.hist[b];
    const int32_t *hsh = wsh + kScratchHeader;
    const uint16_t *lst = (const uint16_t *)(hsh + max_nbins);
    T s[4] = {0, 0, 0, 0}, st = 0;
#pragma unroll 2
    for (int t = lane; t < nd; t += 32) {
        const int j = lst[t];
        const int Lj = hsh[j];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (cand[c] != kNoLabel) s[c] += min((T)hist[hidx(im, cand[c], j)] * m, (T)Lj * sz[c]);
        st += min((T)(hist[hidx(im, k, j)] - Lj) * m, (T)Lj * s_rest);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (cand[c] != kNoLabel) S[c] = warp_sum(s[c]);  // the same slots are empty on every lane
    S_st = warp_sum(st);
}

// Replay a large block's move into buffer `buf` (whole warp).
__device__ void replay_large_block(const DevImage &im, int buf, int level, int bx, int by, uint32_t d, int lane,
                                   int32_t *wsh, int max_nbins)
{
    const int k = (int)(d >> 16), n = (int)(d & 0xFFFFu);
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    const int m = (x1 - x0) * (y1 - y0);
    const int nd = block_sparse_hist(im, x0, x1, y0, y1, lane, wsh, max_nbins);
    block_sparse_apply_clear(im, buf, k, n, nd, lane, wsh, max_nbins);
    if (lane == 0) {
        im.lab[level][buf][SEEDS_IDX(im, by * im.nbx[level] + bx, (int64_t)im.nbx[level] * im.nby[level])] =
            (uint16_t)SEEDS_IDX(im, n, im.K);
        move_size(im, buf, k, n, m);
        if (im.prior) move_xy(im, buf, k, n, x0, x1, y0, y1);
    }
}

__device__ uint32_t judge_large_block_c(const DevImage &im, int b, int nb, int level, int bx, int by, int k,
                                        const int cand[4], int x0, int x1, int y0, int y1, int lane, int32_t *wsh,
                                        int max_nbins);

// Unit (ux,uy) of the union lattice, one warp: replay the previous phase's
// move of that unit (cphase >= 0), then judge this phase's unit.
__device__ void op_block_phase_warp(const DevImage &im, int o, int level, int phase, int cphase, int units, int u,
                                    int lane, int32_t *wsh, int max_nbins)
{
    if (u >= units) return;
    const int b = o & 1, nb = b ^ 1;
    const int nx = im.nbx[level], ny = im.nby[level];
    int mcols, mrows, ncols, nrows;
    lattice(nx, ny, phase, cphase, &mcols, &mrows);
    lattice(nx, ny, phase, -1, &ncols, &nrows);
    const int uy = u / mcols, ux = u - uy * mcols;
    if (cphase >= 0) {
        int ccols, crows;
        lattice(nx, ny, cphase, -1, &ccols, &crows);
        if (ux < ccols && uy < crows) {
            const uint32_t d = im.dec[nb][SEEDS_IDX(im, uy * ccols + ux, im.units_cap)];
            if (d != kNoMove) {
                replay_large_block(im, nb, level, 2 * ux + (cphase & 1), 2 * uy + (cphase >> 1), d, lane, wsh,
                                   max_nbins);
                if (lane == 0) im.dec[nb][SEEDS_IDX(im, uy * ccols + ux, im.units_cap)] = kNoMove;
            }
        }
    }
    if (ux >= ncols || uy >= nrows) return;
    const int uu = uy * ncols + ux;
    const int bx = 2 * ux + (phase & 1), by = 2 * uy + (phase >> 1);
    const uint16_t *lab = im.lab[level][b];
    // the block's extent is read with its labels: fewer dependent trips to L2
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    const int k = lab[by * nx + bx];
    int cand[4];
    const int nc = unit_candidates(lab, nx, ny, bx, by, k, cand);
    const uint32_t d = nc == 0 ? kNoMove
                               : judge_large_block_c(im, b, nb, level, bx, by, k, cand, x0, x1, y0, y1, lane, wsh,
                                                     max_nbins);
    if (lane == 0 && d != kNoMove) im.dec[b][SEEDS_IDX(im, uu, im.units_cap)] = d;
}

// Judge large block (bx,by) of label k that may leave, with candidates cand
// (ascending, kNoLabel in empty slots), the whole warp: the block's sparse
// histogram in the warp's scratch, the intersection sums of Prop. 1, the
// move applied to buffer nb.  Returns the decision (the same on every lane).
__device__ uint32_t judge_large_block_c(const DevImage &im, int b, int nb, int level, int bx, int by, int k,
                                        const int cand[4], int x0, int x1, int y0, int y1, int lane, int32_t *wsh,
                                        int max_nbins)
{
    const int nx = im.nbx[level];
    // the sizes are read before the histogram build: fewer dependent trips to L2
    const int32_t *size = im.size[b];
    int32_t sz[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sz[c] = cand[c] != kNoLabel ? size[SEEDS_IDX(im, cand[c], im.K)] : 1;
    const int m = (x1 - x0) * (y1 - y0);
    const int32_t s_k = size[SEEDS_IDX(im, k, im.K)], s_rest = s_k - m;
    const int nd = block_sparse_hist(im, x0, x1, y0, y1, lane, wsh, max_nbins);
    int64_t S[4] = {0, 0, 0, 0}, S_st = 0;
    // every sum is at most |L| * N: in 32 bits when that fits (the branch
    // is the warp's: m is the block's)
    if ((int64_t)m * im.W * im.H < (1ll << 31))
        warp_block_sums<int32_t>(im, b, wsh, max_nbins, nd, lane, k, cand, sz, s_rest, m, S, S_st);
    else
        warp_block_sums<int64_t>(im, b, wsh, max_nbins, nd, lane, k, cand, sz, s_rest, m, S, S_st);
    // every lane holds the same sums, so every lane takes the same decision;
    // ascending candidates, strictly better replaces: ties to the smallest label
    int n = kNoLabel;
    int64_t Sb = 0, zb = 1;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (cand[c] != kNoLabel && (n == kNoLabel || S[c] * zb > Sb * sz[c])) {
            n = cand[c];
            Sb = S[c];
            zb = sz[c];
        }
    const bool moves = Sb * s_rest > S_st * zb;
    block_sparse_apply_clear(im, nb, moves ? k : -1, n, nd, lane, wsh, max_nbins);
    if (lane == 0 && moves) {
        im.lab[level][nb][SEEDS_IDX(im, by * nx + bx, (int64_t)nx * im.nby[level])] = (uint16_t)SEEDS_IDX(im, n, im.K);
        move_size(im, nb, k, n, m);
        if (im.prior) move_xy(im, nb, k, n, x0, x1, y0, y1);
    }
    return moves ? (((uint32_t)k << 16) | (uint32_t)n) : kNoMove;
}

// ---------------------------------------------------------------------------
// block phase in warp tiles (steps with many units)
// ---------------------------------------------------------------------------

// One warp-tile of a block phase on a level of warp-judged blocks: units
// (ux, uy) of the phase's parity class on the level's block grid, ux in a
// 32-wide column range (one per lane), uy in a kBlockTileUY-row range, as in
// the pixel tile.  The block labels of the tile and a 2-cell halo are staged
// in shared memory; the warp replays the previous phase's moves of the same
// unit positions (cphase >= 0), marks the units that sit on a boundary and
// may leave (from shared memory), decides "stay" for the others, and judges
// the marked blocks one after another (sparse histogram in its scratch).
// The moves and decisions are the ones the per-unit ops take.
__device__ __forceinline__ void op_block_tile(const DevImage &im, int o, int level, int phase, int cphase, int tiles,
                                              int tile, int lane, int32_t *wsh, uint16_t *tsh, int max_nbins)
{
    constexpr int UY = kBlockTileUY;
    if (tile >= tiles) return;
    const int b = o & 1, nb = b ^ 1;
    const int nx = im.nbx[level], ny = im.nby[level];
    const int px = phase & 1, py = phase >> 1;
    const int ncols = (nx - px + 1) >> 1, nrows = (ny - py + 1) >> 1;
    int mcols, mrows;
    lattice(nx, ny, phase, cphase, &mcols, &mrows);
    const int tiles_x = (mcols + kTileUX - 1) / kTileUX;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int ux = tx * kTileUX + lane, uy0 = ty * UY;

    // the previous phase's decisions for the same unit positions
    uint32_t cd[UY];
    int ccols = 0, crows = 0, cpx = 0, cpy = 0;
    if (cphase >= 0) {
        cpx = cphase & 1;
        cpy = cphase >> 1;
        ccols = (nx - cpx + 1) >> 1;
        crows = (ny - cpy + 1) >> 1;
    }
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        const int uy = uy0 + r;
        cd[r] = (ux < ccols && uy < crows) ? im.dec[nb][SEEDS_IDX(im, uy * ccols + ux, im.units_cap)] : kNoMove;
    }
    constexpr int TH = tile_h(UY);
    TileRegs<TH> stage;
    tile_load<TH>(stage, im.lab[level][b], nx, ny, 2 * tx * kTileUX + px - 2, 2 * uy0 + py - 2, lane);
    __syncwarp();  // keeps the loads above the stores
    tile_store<TH>(stage, tsh, lane);

    // replay the previous phase's moves into buffer nb (the staged labels
    // are buffer b's), a block at a time by the whole warp
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        unsigned m = __ballot_sync(0xffffffffu, cd[r] != kNoMove);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t d = __shfl_sync(0xffffffffu, cd[r], l);
            replay_large_block(im, nb, level, 2 * (tx * kTileUX + l) + cpx, 2 * (uy0 + r) + cpy, d, lane, wsh,
                               max_nbins);
        }
        if (cd[r] != kNoMove) im.dec[nb][SEEDS_IDX(im, (uy0 + r) * ccols + ux, im.units_cap)] = kNoMove;
    }
    __syncwarp();

    // boundary units that may leave; the others decide "stay" here
    unsigned mine = 0;
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        const int uy = uy0 + r;
        if (ux < ncols && uy < nrows) {
            const uint16_t *T = tsh + (2 * r + 2) * kTileW + (2 * lane + 2);
            if (may_leave([&](int dx, int dy) { return (int)T[dy * kTileW + dx]; }, (int)T[0]))
                mine |= 1u << r;
        }
    }

    // the warp judges the marked blocks one after another
#pragma unroll
    for (int r = 0; r < UY; ++r) {
        unsigned m = __ballot_sync(0xffffffffu, (mine >> r) & 1u);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const int uxe = tx * kTileUX + l, uy = uy0 + r;
            const int bx = 2 * uxe + px, by = 2 * uy + py;
            const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
            const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
            const uint16_t *T = tsh + (2 * r + 2) * kTileW + (2 * l + 2);
            const int k = T[0];
            int cand[4];
            sorted_candidates(T[-1], T[1], T[-kTileW], T[kTileW], k, cand);
            const uint32_t d =
                judge_large_block_c(im, b, nb, level, bx, by, k, cand, x0, x1, y0, y1, lane, wsh, max_nbins);
            if (lane == 0 && d != kNoMove) im.dec[b][SEEDS_IDX(im, uy * ncols + uxe, im.units_cap)] = d;
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// catch-up: replay op o-1's moves into the buffer that op read
// ---------------------------------------------------------------------------

// A catch-up entry of its own (before a descent, or beside a phase of a step
// that does not fuse replays): replay op o-1's moves into the buffer that op
// read.  `units`: the phase's units; `lanes`: the entry's units.  group 32:
// warp w replays unit w.  Otherwise lane l of warp w reads the decisions of
// units per * 32 * w + 32 * r + l (r < per, coalesced), per = kCatchupPerLane
// when the entry has fewer lanes than units, else 1.
__device__ void op_catchup(const DevImage &im, int o, int level, int phase, int units, int lanes, int group, int off,
                           int lane, int32_t *wsh, int max_nbins)
{
    const int nb = (o & 1) ^ 1;  // = (o-1) & 1: the buffer op o-1 read and decided into
    const int nx = im.nbx[level];
    if (group == 32) {  // large blocks: one warp per unit
        const int u = off >> 5;
        if (u >= units) return;
        const uint32_t d = im.dec[nb][SEEDS_IDX(im, u, im.units_cap)];
        if (d == kNoMove) return;
        int bx, by;
        unit_pos(u, phase, nx, &bx, &by);
        replay_large_block(im, nb, level, bx, by, d, lane, wsh, max_nbins);
        if (lane == 0) im.dec[nb][SEEDS_IDX(im, u, im.units_cap)] = kNoMove;
        return;
    }
    const int per = lanes < units ? kCatchupPerLane : 1;
    const int u0 = (off >> 5) * 32 * per + lane;
    uint32_t d[kCatchupPerLane];
#pragma unroll
    for (int r = 0; r < kCatchupPerLane; ++r) {
        const int u = u0 + 32 * r;
        d[r] = r < per && u < units ? im.dec[nb][SEEDS_IDX(im, u, im.units_cap)] : kNoMove;
        if (d[r] != kNoMove) im.dec[nb][SEEDS_IDX(im, u, im.units_cap)] = kNoMove;
    }
    if (level == 0) {  // pixels
        const bool means = op_at(im.L, im.iters, im.means_iters, o - 1).kind == OP_MPHASE;
#pragma unroll
        for (int r = 0; r < kCatchupPerLane; ++r) {
            if (d[r] == kNoMove) continue;
            int x, y;
            unit_pos(u0 + 32 * r, phase, im.W, &x, &y);
            if (means) {
                replay_pixel(im, nb, y * im.W + x, d[r]);
                move_sums(im, nb, (int)(d[r] >> 16), (int)(d[r] & 0xFFFFu), x, y);
            } else {  // the new label from the named neighbour in the buffer op o reads
                const int dir = (int)(d[r] >> 12) & 3;
                const int qx = x + (dir == 0 ? -1 : dir == 1 ? 1 : 0), qy = y + (dir == 2 ? -1 : dir == 3 ? 1 : 0);
                replay_pixel_dec(im, nb, x, y, d[r], im.lab[0][nb ^ 1][SEEDS_IDX(im, qy * im.W + qx, (int64_t)im.W * im.H)]);
            }
        }
        return;
    }
    if (level_group(im, level) == 32) {  // blocks a warp judges: the warp replays each move (per is 1)
        unsigned m = __ballot_sync(0xffffffffu, d[0] != kNoMove);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t dl = __shfl_sync(0xffffffffu, d[0], l);
            int bx, by;
            unit_pos(u0 - lane + l, phase, nx, &bx, &by);
            replay_large_block(im, nb, level, bx, by, dl, lane, wsh, max_nbins);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kCatchupPerLane; ++r) {  // small blocks: a lane each
        if (d[r] == kNoMove) continue;
        int bx, by;
        unit_pos(u0 + 32 * r, phase, nx, &bx, &by);
        replay_small_block(im, nb, level, bx, by, d[r]);
    }
}

// ---------------------------------------------------------------------------
// descent, output
// ---------------------------------------------------------------------------

// level `level` -> level-1 (both buffers); the finer grid splits each block
// 2x2.  A thread writes kRowChunk consecutive cells of one row of the finer
// grid (pixels at the last descent), with one 16-byte store per buffer where
// the row allows it.
__device__ void op_descend(const DevImage &im, int o, int level, int units, int c)
{
    if (c >= units) return;
    const int t = level - 1;
    const uint16_t *src = im.lab[level][o & 1];
    const int nx = im.nbx[t];  // W at the pixel level
    const int cpr = (nx + kRowChunk - 1) / kRowChunk;
    const int y = c / cpr, x0 = (c - y * cpr) * kRowChunk;
    uint16_t v[kRowChunk];
    if (t >= 1) {  // cell (x, y) of the finer grid lies in cell (x/2, y/2)
        const uint16_t *row = src + (y >> 1) * im.nbx[level];
#pragma unroll
        for (int q = 0; q < kRowChunk; ++q) v[q] = x0 + q < nx ? row[(x0 + q) >> 1] : 0;
    } else {
        // level-1 block bx holds x iff floor(bx*W/n) <= x < floor((bx+1)*W/n);
        // the next pixel steps into the next block when (bx+1)*W < (x+1)*n
        // (every product is below 2^31: W, H, n <= 32768)
        const int W = nx, n1x = im.nbx[1], n1y = im.nby[1];
        const int by = ((y + 1) * n1y - 1) / im.H;
        int bx = ((x0 + 1) * n1x - 1) / W;
        const uint16_t *row = src + by * n1x;
#pragma unroll
        for (int q = 0; q < kRowChunk; ++q) {
            if (q > 0 && (bx + 1) * W < (x0 + q + 1) * n1x) ++bx;
            v[q] = row[min(bx, n1x - 1)];
        }
    }
    uint16_t *d0 = im.lab[t][0] + (int64_t)y * nx + x0, *d1 = im.lab[t][1] + (int64_t)y * nx + x0;
    if (nx % kRowChunk == 0) {  // whole chunks, rows 16-byte aligned
        const uint4 w = make_uint4(v[0] | (uint32_t)v[1] << 16, v[2] | (uint32_t)v[3] << 16,
                                   v[4] | (uint32_t)v[5] << 16, v[6] | (uint32_t)v[7] << 16);
        *(uint4 *)d0 = w;
        *(uint4 *)d1 = w;
        return;
    }
#pragma unroll
    for (int q = 0; q < kRowChunk; ++q)
        if (x0 + q < nx) d0[q] = d1[q] = v[q];
}

// int32 labels: a thread converts kRowChunk consecutive pixels of a row
// (one 16-byte load, two 16-byte stores where the row allows it)
__device__ void op_output(const DevImage &im, int o, int units, int c)
{
    if (c >= units) return;
    const int W = im.W, cpr = (W + kRowChunk - 1) / kRowChunk;
    const int y = c / cpr, x0 = (c - y * cpr) * kRowChunk;
    const uint16_t *lab = im.lab[0][o & 1] + (int64_t)y * W;
    int32_t *out = im.out + (int64_t)y * W;
    if (W % kRowChunk == 0 && ((uintptr_t)im.out & 15) == 0) {
        const uint4 v = *(const uint4 *)(lab + x0);
        *(int4 *)(out + x0) = make_int4(v.x & 0xFFFF, v.x >> 16, v.y & 0xFFFF, v.y >> 16);
        *(int4 *)(out + x0 + 4) = make_int4(v.z & 0xFFFF, v.z >> 16, v.w & 0xFFFF, v.w >> 16);
        return;
    }
#pragma unroll
    for (int q = 0; q < kRowChunk; ++q)
        if (x0 + q < W) out[x0 + q] = lab[x0 + q];
}

// Anytime termination (Sec. 5.4): every image whose output op has not run
// gets its partition after op o, the last op the grid completed.  Its labels
// live on the grid of the level it stands at (a phase: that level; a
// descent from l: level l-1; the init: level L), in buffer (o+1)&1, and each
// pixel takes the label of the unit that holds it: unit column
// bx = ((x+1)*nbx - 1) / W inverts the edges floor(i*W/nbx), rows likewise.
// Few images: every thread walks each image; many: a block per image.
__device__ __noinline__ void anytime_output(const DevImage *imgs, int nimg, int o)
{
    const bool per_block = nimg >= (int)gridDim.x;
    const int i0 = per_block ? blockIdx.x : 0, istep = per_block ? gridDim.x : 1;
    const int64_t t0 = per_block ? threadIdx.x : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tstep = per_block ? blockDim.x : (int64_t)gridDim.x * blockDim.x;
    for (int i = i0; i < nimg; i += istep) {
        const DevImage &im = imgs[i];
        if (o >= num_ops(im.L, im.iters, im.means_iters) - 1) continue;  // finished: its output ran
        const OpDesc d = op_at(im.L, im.iters, im.means_iters, o);
        const int level = d.kind == OP_PHASE      ? d.level
                          : d.kind == OP_DESCEND  ? d.level - 1
                          : d.kind == OP_INIT     ? im.L
                                                  : 0;  // the means iterations run on pixels
        const uint16_t *lab = im.lab[level][(o + 1) & 1];
        const int W = im.W, nx = im.nbx[level], ny = im.nby[level];
        const int64_t npx = (int64_t)W * im.H;
        for (int64_t p = t0; p < npx; p += tstep) {
            const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
            int v;
            if (level == 0) {
                v = lab[p];
            } else {
                const int bx = (int)(((int64_t)(x + 1) * nx - 1) / W);
                const int by = (int)(((int64_t)(y + 1) * ny - 1) / im.H);
                v = lab[by * nx + bx];
            }
            im.out[p] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

// Up to 1024 threads per CTA, with registers capped at 64 per thread so that
// a whole SM's worth of warps (2048 threads) stays resident.
__global__ void __launch_bounds__(1024, 1) seeds_persistent(const DevImage *__restrict__ imgs, Schedule S,
                                                        GridBarrier *bar, int32_t *err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps_blk = blockDim.x >> 5;

    // per-warp scratch sized for the largest histogram of the context
    const int wbytes = warp_scratch_bytes(S.max_nbins);
    int32_t *wsh = (int32_t *)(smem + (size_t)warp * wbytes);
    uint16_t *tsh = (uint16_t *)(smem + (size_t)warp * wbytes + warp_hist_scratch_bytes(S.max_nbins));
    for (int i = lane; i < wbytes / 4; i += 32) wsh[i] = 0;
    __syncwarp();

    // A step's virtual warps are dealt to the CTAs in rounds: round r gives
    // CTA c the nwarps_blk virtual warps from (r * gridDim.x + c) * nwarps_blk
    // on.  Warp w takes the w-th of round 0; after that the CTA's warps take
    // its next one from a shared counter as they finish, so one slow unit
    // does not hold up the units queued behind it on the same warp.  Two
    // counters alternate between steps; the grid barrier's CTA barrier
    // orders each reset before its use.  A step that fits in one round is
    // dealt round-robin instead (virtual warp w * gridDim.x + c to warp w of
    // CTA c), so that its warps spread over every SM rather than filling the
    // first CTAs.
    __shared__ unsigned s_next[2];
    if (threadIdx.x == 0) s_next[0] = s_next[1] = 0;
    __syncthreads();
    // values that live through every step are kept few: the grid's warp
    // count and the CTA's first warp are 32-bit (a grid has fewer than 2^31
    // warps) and the anytime start time waits in shared memory
    const int nwarps = (int)gridDim.x * nwarps_blk;
    const int cta_first = (int)blockIdx.x * nwarps_blk;
    const bool tracer = S.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
    if (tracer) S.trace[0] = global_ns();
    const bool anytime = S.stop_steps > 0 || S.budget_ns > 0;
    __shared__ uint64_t s_t_start;
    if (threadIdx.x == 0) s_t_start = anytime ? global_ns() : 0;  // read by thread 0 only

    for (int s = 0; s < S.nsteps; ++s) {
        const int e0 = S.step_first[s], e1 = S.step_first[s + 1];
        const int64_t total = S.step_vt[s];
        if (threadIdx.x == 0) s_next[(s + 1) & 1] = 0;
        const bool rounds = (int64_t)nwarps * 32 < total;  // work beyond round 0 for some CTA
        // odd steps walk the step's units from the end, so a step starts on
        // the images whose state the step before touched last (still in L2)
        const bool reverse = (s & 1) != 0;
        for (unsigned i = warp;; ) {
            const int64_t fwd = rounds ? ((int64_t)(i / nwarps_blk) * nwarps + cta_first + (i % nwarps_blk)) * 32
                                       : ((int64_t)i * gridDim.x + blockIdx.x) * 32;
            if (fwd >= total) break;
            const int64_t base = reverse ? total - 32 - fwd : fwd;
            int lo = e0, hi = e1 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.ent[mid].vt_begin <= base)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const StepEntry E = S.ent[lo];
            const DevImage &im = imgs[E.img];
            const int off = (int)(base - E.vt_begin);
            switch (E.op) {
            case OP_INIT:
                op_init(im, off >> 5, lane, wsh);
                break;
            case OP_PHASE:
                if (E.level == 0)
                    if (im.tile_uy == 2)
                        op_pixel_tile<false, 2>(im, E.opidx, E.phase, E.cphase, E.units, off >> 5, lane, tsh);
                    else
                        op_pixel_tile<false, kTileUY>(im, E.opidx, E.phase, E.cphase, E.units, off >> 5, lane, tsh);
                else if (E.group == 1)
                    op_block_phase_thread(im, E.opidx, E.level, E.phase, E.cphase, E.units, off + lane);
                else
                    op_block_phase_warp(im, E.opidx, E.level, E.phase, E.cphase, E.units, off >> 5, lane, wsh,
                                        S.max_nbins);
                break;
            case OP_BTILE:
                op_block_tile(im, E.opidx, E.level, E.phase, E.cphase, E.units, off >> 5, lane, wsh, tsh, S.max_nbins);
                break;
            case OP_MPHASE:
                op_means_tile(im, E.opidx, E.phase, E.cphase, E.units, off >> 5, lane, tsh);
                break;
            case OP_MINIT:
                op_means_init(im, E.opidx, E.units, off + lane, lane);
                break;
            case OP_CATCHUP:
                op_catchup(im, E.opidx, E.level, E.phase, (int)phase_units(im, E.level, E.phase), E.units, E.group,
                           off, lane, wsh, S.max_nbins);
                break;
            case OP_DESCEND:
                op_descend(im, E.opidx, E.level, E.units, off + lane);
                break;
            case OP_OUTPUT:
                op_output(im, E.opidx, E.units, off + lane);
                break;
            default:
                break;
            }
            if (!rounds) break;
            unsigned nx = 0;
            if (lane == 0) nx = atomicAdd(&s_next[s & 1], 1u);
            i = __shfl_sync(0xffffffffu, nx, 0) + nwarps_blk;
        }
        if (s + 1 < S.nsteps) {
            if (!anytime) {
                if (!grid_sync_count(bar, err, (unsigned)(s + 1) * gridDim.x,
                                     S.timeout_ns ? S.timeout_ns : kBarrierTimeoutNs,
                                     blockIdx.x != 0 || S.withhold != s + 1))
                    return;
            } else {
                const bool want_stop = threadIdx.x == 0 && ((S.stop_steps > 0 && s + 1 >= S.stop_steps) ||
                                                            (S.budget_ns > 0 && global_ns() - s_t_start >= S.budget_ns));
                const int go = grid_sync(bar, err, want_stop, S.timeout_ns ? S.timeout_ns : kBarrierTimeoutNs,
                                         blockIdx.x != 0 || S.withhold != s + 1);
                if (go == 0) return;
                if (go == 2) {
                    anytime_output(imgs, S.nimg, s);
                    if (blockIdx.x == 0 && threadIdx.x == 0 && S.steps_out) *S.steps_out = s + 1;
                    return;
                }
            }
        }
        if (tracer) S.trace[1 + s] = global_ns();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && S.steps_out) *S.steps_out = S.nsteps;
}

__global__ void set_io_kernel(DevImage *imgs, IoChunk chunk)
{
    const int i = threadIdx.x;
    if (i < chunk.n) {
        DevImage &im = imgs[chunk.first + i];
        im.rgb = chunk.e[i].rgb;
        im.stride = chunk.e[i].stride;
        im.out = chunk.e[i].out;
    }
}

// recount an image's histograms (both buffers) from the labels of one level
// of buffer 0 (test hook)
__global__ void recount_kernel(const DevImage *imgs, int img, int level, int64_t npix, int zero_pass)
{
    const DevImage &im = imgs[img];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (zero_pass) {
        const int64_t nh = (int64_t)im.K * im.nbins;
        for (int64_t t = i; t < nh; t += stride) im.hist[0][t] = im.hist[1][t] = 0;
        for (int64_t t = i; t < im.K; t += stride) im.size[0][t] = im.size[1][t] = 0;
        if (im.prior)  // the compactness prior's coordinate sums
            for (int64_t t = i; t < (int64_t)im.K * 5; t += stride) im.msum[0][t] = im.msum[1][t] = 0;
        return;
    }
    if (i >= npix) return;
    const int y = (int)(i / im.W), x = (int)(i - (int64_t)y * im.W);
    int k;
    if (level == 0) {
        k = im.lab[0][0][i];
    } else {
        const int nx = im.nbx[level], ny = im.nby[level];
        const int bx = (int)(((int64_t)(x + 1) * nx - 1) / im.W);
        const int by = (int)(((int64_t)(y + 1) * ny - 1) / im.H);
        k = im.lab[level][0][by * nx + bx];
    }
    const int j = bin_at(im, (int)i);
    atomicAdd(&im.hist[0][hidx(im, k, j)], 1);
    atomicAdd(&im.hist[1][hidx(im, k, j)], 1);
    atomicAdd(&im.size[0][k], 1);
    atomicAdd(&im.size[1][k], 1);
    if (im.prior)
        for (int q = 0; q < 2; ++q) {
            atomicAdd(&im.msum[q][(int64_t)k * 5 + 3], (unsigned long long)x);
            atomicAdd(&im.msum[q][(int64_t)k * 5 + 4], (unsigned long long)y);
        }
}

// ---------------------------------------------------------------------------
// serving: install an admitted image, build an epoch's schedule
// ---------------------------------------------------------------------------

// the slot's record, and the block edge tables of every level
__global__ void admit_kernel(DevImage *imgs, int slot, DevImage rec)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) imgs[slot] = rec;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int l = 1; l <= rec.L; ++l) {
        int32_t *xe = (int32_t *)rec.xe[l], *ye = (int32_t *)rec.ye[l];
        for (int i = t; i <= rec.nbx[l]; i += nt) xe[i] = (int32_t)((int64_t)i * rec.W / rec.nbx[l]);
        for (int i = t; i <= rec.nby[l]; i += nt) ye[i] = (int32_t)((int64_t)i * rec.H / rec.nby[l]);
    }
}

// One block, a thread per step: count the step's entries, scan, write them.
__global__ void epoch_schedule_kernel(const DevImage *imgs, EpochPlan plan, StepEntry *ent, int32_t *first,
                                      int64_t *vt)
{
    __shared__ int32_t cnt[1024];
    const int s = threadIdx.x;
    StepEntry tmp[2];
    int c = 0;
    int fuse = 2;
    if (s < plan.nsteps) {
        int64_t sized[2] = {0, 0};  // the step's size with fused per-unit entries, with fused tiles
        for (int pass = 0; pass < 3; ++pass) {
            int64_t v = 0;
            const int mode = pass == 0 ? 2 : pass == 1 ? 2 | kWideStep : fuse;
            for (int i = 0; i < plan.n; ++i) {
                const EpochSlot &q = plan.s[i];
                const int o = q.begin + s;
                if (o >= q.end) continue;
                const DevImage &im = imgs[q.slot];
                const bool cu =
                    s == 0 ? q.catchup != 0 : is_phase(op_at(im.L, im.iters, im.means_iters, o - 1).kind);
                const int m = emit_entries(im, q.slot, o, cu, mode, tmp, &v);
                if (pass == 2) c += m;
            }
            if (pass < 2) sized[pass] = v;
            if (pass == 1) fuse = step_mode(sized[0], sized[1], plan.split_below, plan.tile_policy);
        }
    }
    cnt[s] = c;
    __syncthreads();
    if (s == 0) {  // exclusive scan over the steps (at most 1024)
        int acc = 0;
        for (int t = 0; t < plan.nsteps; ++t) {
            const int v = cnt[t];
            cnt[t] = acc;
            acc += v;
        }
        first[plan.nsteps] = acc;
    }
    __syncthreads();
    if (s >= plan.nsteps) return;
    int e = cnt[s];
    first[s] = e;
    int64_t v = 0;
    for (int i = 0; i < plan.n; ++i) {
        const EpochSlot &q = plan.s[i];
        const int o = q.begin + s;
        if (o >= q.end) continue;
        const DevImage &im = imgs[q.slot];
        const bool cu = s == 0 ? q.catchup != 0 : is_phase(op_at(im.L, im.iters, im.means_iters, o - 1).kind);
        e += emit_entries(im, q.slot, o, cu, fuse, ent + e, &v);
    }
    vt[s] = v;
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

cudaError_t launch_admit(DevImage *d_imgs, int slot, const DevImage &rec, cudaStream_t s)
{
    admit_kernel<<<4, 256, 0, s>>>(d_imgs, slot, rec);
    return cudaGetLastError();
}

cudaError_t launch_epoch_schedule(const DevImage *d_imgs, const EpochPlan &plan, StepEntry *ent, int32_t *first,
                                  int64_t *vt, cudaStream_t s)
{
    if (plan.nsteps < 1 || plan.nsteps > 1024) return cudaErrorInvalidValue;
    epoch_schedule_kernel<<<1, 1024, 0, s>>>(d_imgs, plan, ent, first, vt);
    return cudaGetLastError();
}

cudaError_t launch_set_io(DevImage *d_imgs, const IoChunk &chunk, cudaStream_t s)
{
    set_io_kernel<<<1, kIoChunk, 0, s>>>(d_imgs, chunk);
    return cudaGetLastError();
}

// The kernel's dynamic shared-memory limit is one attribute per function and
// device, shared by every context, server and static call in the process:
// it is only ever raised, never lowered, so a launch configured for a large
// histogram stays valid after a smaller one configures its own.  The current
// value is read back each time, so a device reset (which clears it) is seen.
cudaError_t prepare_persistent(size_t smem)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, seeds_persistent);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(seeds_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t persistent_max_blocks_per_sm(int threads, size_t smem, int *n)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, seeds_persistent, threads, smem);
}

cudaError_t upload_lab_tables(cudaStream_t s)
{
    static std::mutex mu;
    static bool done[64] = {};
    static bool built = false;
    static int32_t lin[256], mq[9];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!built) {
        // sRGB decoding curve (IEC 61966-2-1) and the sRGB -> XYZ (D65) matrix
        static const double m[3][3] = {{0.4124, 0.3576, 0.1805}, {0.2126, 0.7152, 0.0722}, {0.0193, 0.1192, 0.9505}};
        for (int v = 0; v < 256; ++v) {
            const double c = v / 255.0;
            const double l = c <= 0.04045 ? c / 12.92 : std::pow((c + 0.055) / 1.055, 2.4);
            lin[v] = (int32_t)std::llround(l * 16777216.0);
        }
        for (int i = 0; i < 3; ++i) {
            const double white = m[i][0] + m[i][1] + m[i][2];
            for (int j = 0; j < 3; ++j) mq[3 * i + j] = (int32_t)std::llround(m[i][j] / white * 1048576.0);
        }
        built = true;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return done[dev] ? cudaSuccess : cudaErrorStreamCaptureUnsupported;
    e = cudaMemcpyToSymbolAsync(g_lab_lin, lin, sizeof(lin), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_lab_m, mq, sizeof(mq), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

cudaError_t launch_persistent(const DevImage *d_imgs, const Schedule &sch, GridBarrier *bar, int32_t *err, int grid,
                              int threads, size_t smem, cudaStream_t s)
{
    seeds_persistent<<<grid, threads, smem, s>>>(d_imgs, sch, bar, err);
    return cudaGetLastError();
}

cudaError_t launch_recount(const DevImage *d_imgs, int img, int level, int64_t npix, cudaStream_t s)
{
    recount_kernel<<<256, 256, 0, s>>>(d_imgs, img, level, npix, 1);
    const int64_t blocks = (npix + 255) / 256;
    recount_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_imgs, img, level, npix, 0);
    return cudaGetLastError();
}

// ===========================================================================
// One image with no allocation at all: every byte of device state lives in a
// file-scope static device array.  For callers that may not allocate device
// memory (see seeds_run_static in seeds.h).
// ===========================================================================

static __device__ __align__(256) unsigned char g_static_scratch[SEEDS_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
unsigned char *g_static_addr[kStaticMaxDevices] = {};

// Host address stand-ins are not device addresses: ask the runtime, with the
// device current.  The lookup allocates nothing; it is repeated on every call
// whose stream is not being captured (so a context the host application
// rebuilt, e.g. after a device reset, is seen) and the last answer for the
// device is kept for calls made during a capture.
cudaError_t static_scratch_address(int dev, cudaStream_t stream, unsigned char **out)
{
    if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone || !g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = (unsigned char *)p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

size_t sal(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// everything the setup kernel needs, passed by value
struct StaticSetup {
    DevImage img;  // pointers already inside the scratch
    StepEntry *ent;
    int32_t *first;
    int64_t *vt;
    unsigned char *zero_begin;  // barrier and error word
    int32_t zero_bytes;
    int32_t nops;
    int32_t split_below;  // fuse_step's threshold in warps
    DevImage *img_out;
};

// Lays out one image inside the scratch: the image record, the block edge
// tables of every level, and the op schedule (one op per step, with the
// catch-up of the previous phase); clears the barrier and the error word.
__global__ void static_setup_kernel(StaticSetup S)
{
    const DevImage &im = S.img;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int l = 1; l <= im.L; ++l) {
        int32_t *xe = (int32_t *)im.xe[l], *ye = (int32_t *)im.ye[l];
        for (int i = t; i <= im.nbx[l]; i += nt) xe[i] = (int32_t)((int64_t)i * im.W / im.nbx[l]);
        for (int i = t; i <= im.nby[l]; i += nt) ye[i] = (int32_t)((int64_t)i * im.H / im.nby[l]);
    }
    for (int i = t; i < S.zero_bytes; i += nt) S.zero_begin[i] = 0;
    if (t != 0) return;
    *S.img_out = im;
    int ne = 0;
    for (int o = 0; o < S.nops; ++o) {
        S.first[o] = ne;
        int64_t vt = 0;
        const bool catchup = o > 0 && is_phase(op_at(im.L, im.iters, im.means_iters, o - 1).kind);
        StepEntry tmp[2];
        int64_t vf = 0, vtile = 0;
        emit_entries(im, 0, o, catchup, 2, tmp, &vf);
        emit_entries(im, 0, o, catchup, 2 | kWideStep, tmp, &vtile);
        ne += emit_entries(im, 0, o, catchup, step_mode(vf, vtile, S.split_below), S.ent + ne, &vt);
        S.vt[o] = vt;
    }
    S.first[S.nops] = ne;
}

__global__ void static_status_kernel(const int32_t *err, int32_t *status) { *status = *err; }

}  // namespace seeds

using namespace seeds;

extern "C" int seeds_run_static(const seeds_params *p, const uint8_t *d_rgb, int64_t row_stride_bytes,
                                int32_t *d_labels_out, int32_t *d_status, void *stream)
{
    // ---- parameters, grid (Sec. 5.1) and the image's state layout: the
    // same heap-free derivation the allocating contexts use
    if (!p || !d_rgb || !d_labels_out) return SEEDS_ERR_INVALID;
    host::ImageCore h;
    int rc = host::derive_core(p, &h, nullptr, nullptr);
    if (rc) return rc;
    if (row_stride_bytes < 3 * (int64_t)p->width) return SEEDS_ERR_INVALID;
    const int nops = h.nops;

    // ---- layout inside the scratch: the image record, the barrier and the
    // error word, the schedule, then the image's state as derive_core laid it out
    size_t off = 0;
    const size_t o_img = off;
    off = sal(off + sizeof(DevImage));
    const size_t o_zero = off, o_bar = off, o_err = off + 16;  // barrier | error word
    off = sal(off + 32);
    const size_t o_ent = off;
    off = sal(off + sizeof(StepEntry) * 2 * (size_t)nops);
    const size_t o_first = off;
    off = sal(off + 4 * (size_t)(nops + 1));
    const size_t o_vt = off;
    off = sal(off + 8 * (size_t)nops);
    const size_t o_state = off;
    off += h.bytes;
    if (off > (size_t)SEEDS_STATIC_SCRATCH_BYTES) return SEEDS_ERR_STATIC_SIZE;
    if (p->color_space == 1 && upload_lab_tables((cudaStream_t)stream) != cudaSuccess) return SEEDS_ERR_CUDA;

    // ---- the scratch's device address on the current device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SEEDS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    if (static_scratch_address(dev, s, &base) != cudaSuccess) return SEEDS_ERR_CUDA;

    StaticSetup S;
    std::memset(&S, 0, sizeof(S));
    const seeds_tuning knobs{0, 0, 0, kSmallMax, kTileUY, 0};
    S.img = host::make_dev_image(h, base + o_state, knobs, IoEntry{d_rgb, row_stride_bytes, d_labels_out},
                                 (int32_t *)(base + o_err));
    S.ent = (StepEntry *)(base + o_ent);
    S.first = (int32_t *)(base + o_first);
    S.vt = (int64_t *)(base + o_vt);
    S.zero_begin = base + o_zero;
    S.zero_bytes = 32;
    S.nops = nops;
    S.img_out = (DevImage *)(base + o_img);

    // ---- launch configuration of the persistent kernel (as a context would):
    // the largest CTA whose warps' shared scratch fits
    int threads = 0, sms = 0, per_sm = 0;
    size_t smem = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SEEDS_ERR_CUDA;
    for (int t : {1024, 512, 256, 128}) {
        smem = (size_t)(t / 32) * warp_scratch_bytes(h.nbins);
        per_sm = 0;
        if (prepare_persistent(smem) == cudaSuccess &&
            persistent_max_blocks_per_sm(t, smem, &per_sm) == cudaSuccess && per_sm >= 1) {
            threads = t;
            break;
        }
        cudaGetLastError();  // a size that does not fit is not an error of the call
    }
    if (threads == 0) return SEEDS_ERR_CUDA;

    S.split_below = sms * 32;
    static_setup_kernel<<<8, 256, 0, s>>>(S);
    if (cudaGetLastError() != cudaSuccess) return SEEDS_ERR_CUDA;
    Schedule sch{};
    sch.ent = S.ent;
    sch.step_first = S.first;
    sch.step_vt = S.vt;
    sch.nsteps = nops;
    sch.max_nbins = h.nbins;
    sch.trace = nullptr;
    if (launch_persistent(S.img_out, sch, (GridBarrier *)(base + o_bar), (int32_t *)(base + o_err), per_sm * sms,
                          threads, smem, s) != cudaSuccess)
        return SEEDS_ERR_CUDA;
    if (d_status) {
        static_status_kernel<<<1, 1, 0, s>>>((const int32_t *)(base + o_err), d_status);
        if (cudaGetLastError() != cudaSuccess) return SEEDS_ERR_CUDA;
    }
    return SEEDS_OK;
}
