// seeds_kernels.cu -- sm_103a kernels of the SEEDS hot path.
//
// One persistent kernel runs a whole schedule (see seeds_device.cuh):
//   op_init        quantise RGB to colour bins (one warp per initial
//                  superpixel rectangle), build its histogram with
//                  warp-aggregated shared-memory atomics, write the grid
//                  labels (Sec. 5.1, Eq. 4)
//   op_*_phase     judge every unit of one parity phase against the state
//                  at phase start and append accepted moves (Sec. 5.2-5.3:
//                  Prop. 1 for blocks, Prop. 1 + Prop. 2 for pixels)
//   apply slot     apply the phase's moves: labels and incremental histogram
//                  updates (Sec. 5.3, "Updating the Color Distributions")
//   op_descend     copy block labels to the next finer grid (Sec. 5.1-5.2,
//                  coarse to fine)
//   op_output      int32 labels for the caller
// Grid barriers between slots spin with a time limit; a barrier that runs
// out sets the error word and every block leaves the kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "seeds_device.cuh"

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

// Grid-wide barrier for a persistent launch whose blocks are all resident.
// Returns false when the wait ran out or another block reported an error.
__device__ bool grid_sync(GridBarrier *bar, int32_t *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g = ld_acquire_u32(&bar->gen);
        __threadfence();
        unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            uint64_t t0 = global_ns();
            while (ld_acquire_u32(&bar->gen) == g) {
                if (ld_relaxed_i32(err) != 0) {
                    ok = 0;
                    break;
                }
                __nanosleep(40);
                if (global_ns() - t0 > kBarrierTimeoutNs) {
                    atomicOr(err, DERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int hidx(const DevImage &im, int k, int j)
{
    return im.hist_jmajor ? j * im.K + k : k * im.nbins + j;
}

__device__ __forceinline__ int bin_at(const DevImage &im, int p)
{
    return im.bins16 ? (int)((const uint16_t *)im.bins)[p] : (int)((const uint8_t *)im.bins)[p];
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
    unsigned prev = ((m << 1) | (m >> 7)) & 0xFFu;  // bit r = bit r-1 of m
    unsigned next = ((m >> 1) | (m << 7)) & 0xFFu;  // bit r = bit r+1 of m
    unsigned starts = m & ~prev;
    unsigned lone_corners = m & ~prev & ~next & 0x55u;
    return __popc(starts) - __popc(lone_corners) == 1;
}

// label of grid cell (x,y) or kNoLabel outside
__device__ __forceinline__ int cell(const uint16_t *lab, int nx, int ny, int x, int y)
{
    return (x < 0 || y < 0 || x >= nx || y >= ny) ? (int)kNoLabel : (int)lab[y * nx + x];
}

// Shared unit logic: boundary test, ring validity, sorted distinct
// candidates.  Returns the candidate count (0 = no move possible).
__device__ __forceinline__ int unit_candidates(const uint16_t *lab, int nx, int ny, int x, int y, int k, int cand[4])
{
    const int lf = cell(lab, nx, ny, x - 1, y), rt = cell(lab, nx, ny, x + 1, y);
    const int up = cell(lab, nx, ny, x, y - 1), dn = cell(lab, nx, ny, x, y + 1);
    const bool boundary = (lf != k && lf != kNoLabel) || (rt != k && rt != kNoLabel) ||
                          (up != k && up != kNoLabel) || (dn != k && dn != kNoLabel);
    if (!boundary) return 0;
    unsigned m = 0;
    m |= (cell(lab, nx, ny, x - 1, y - 1) == k) << 0;
    m |= (up == k) << 1;
    m |= (cell(lab, nx, ny, x + 1, y - 1) == k) << 2;
    m |= (rt == k) << 3;
    m |= (cell(lab, nx, ny, x + 1, y + 1) == k) << 4;
    m |= (dn == k) << 5;
    m |= (cell(lab, nx, ny, x - 1, y + 1) == k) << 6;
    m |= (lf == k) << 7;
    if (!ring_allows_leaving(m)) return 0;
    // sort the four neighbour labels (kNoLabel sorts last), then keep the
    // distinct ones other than k
    int a = lf, b = rt, c = up, d = dn, t;
#define SEEDS_CSWAP(p, q) \
    if (p > q) {          \
        t = p;            \
        p = q;            \
        q = t;            \
    }
    SEEDS_CSWAP(a, b) SEEDS_CSWAP(c, d) SEEDS_CSWAP(a, c) SEEDS_CSWAP(b, d) SEEDS_CSWAP(b, c)
#undef SEEDS_CSWAP
    int nc = 0, last = -1;
    const int v[4] = {a, b, c, d};
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (v[i] != kNoLabel && v[i] != k && v[i] != last) {
            cand[nc++] = v[i];
            last = v[i];
        }
    return nc;
}

// append one move per lane that has one (whole warp calls this)
__device__ __forceinline__ void append_moves_warp(const DevImage &im, int s, bool has, uint32_t w0, uint32_t w1,
                                                  int lane, int32_t *err)
{
    unsigned ballot = __ballot_sync(0xffffffffu, has);
    if (!ballot) return;
    int leader = __ffs(ballot) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&im.cnt[s & 1], __popc(ballot));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (has) {
        int idx = base + __popc(ballot & ((1u << lane) - 1u));
        if (idx < im.moves_cap) {
            im.moves[2 * idx] = w0;
            im.moves[2 * idx + 1] = w1;
        } else {
            atomicOr(err, DERR_BOUNDS);
        }
    }
}

__device__ __forceinline__ void append_move_single(const DevImage &im, int s, uint32_t w0, uint32_t w1, int32_t *err)
{
    int idx = atomicAdd(&im.cnt[s & 1], 1);
    if (idx < im.moves_cap) {
        im.moves[2 * idx] = w0;
        im.moves[2 * idx + 1] = w1;
    } else {
        atomicOr(err, DERR_BOUNDS);
    }
}

// ---------------------------------------------------------------------------
// op_init: one warp per initial superpixel rectangle
// ---------------------------------------------------------------------------

__device__ void op_init(const DevImage &im, int k, int lane, int32_t *wsh)
{
    if (k >= im.K) return;
    const int sx = k % im.gx, sy = k / im.gx;
    const int x0 = (int)((int64_t)sx * im.W / im.gx), x1 = (int)((int64_t)(sx + 1) * im.W / im.gx);
    const int y0 = (int)((int64_t)sy * im.H / im.gy), y1 = (int)((int64_t)(sy + 1) * im.H / im.gy);
    const int rw = x1 - x0, area = rw * (y1 - y0);
    const int B = im.B;
    for (int base = 0; base < area; base += 32) {
        const int t = base + lane;
        const bool act = t < area;
        int j = -1;
        if (act) {
            const int dy = t / rw, x = x0 + (t - dy * rw), y = y0 + dy;
            const uint8_t *px = im.rgb + (int64_t)y * im.stride + 3 * (int64_t)x;
            const int r = px[0], g = px[1], b = px[2];
            j = ((r * B) >> 8) * B * B + ((g * B) >> 8) * B + ((b * B) >> 8);
            const int p = y * im.W + x;
            if (im.bins16)
                ((uint16_t *)im.bins)[p] = (uint16_t)j;
            else
                ((uint8_t *)im.bins)[p] = (uint8_t)j;
            if (im.L == 0) im.lab[0][p] = (uint16_t)k;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, j);
        if (act && lane == __ffs(peers) - 1) atomicAdd(&wsh[j], __popc(peers));
    }
    __syncwarp();
    for (int j = lane; j < im.nbins; j += 32) {
        im.hist[hidx(im, k, j)] = wsh[j];
        wsh[j] = 0;
    }
    __syncwarp();
    if (lane == 0) im.size[k] = area;
    if (im.L >= 1 && lane < 4) {
        const int L = im.L;
        const int bx = 2 * sx + (lane & 1), by = 2 * sy + (lane >> 1);
        im.lab[L][by * im.nbx[L] + bx] = (uint16_t)k;
    }
}

// ---------------------------------------------------------------------------
// pixel phase: one thread per pixel of the parity class
// ---------------------------------------------------------------------------

__device__ void op_pixel_phase(const DevImage &im, int phase, int units, int s, int u, int lane, int32_t *err)
{
    bool has = false;
    uint32_t w0 = 0, w1 = 0;
    if (u < units) {
        const int px = phase & 1, py = phase >> 1;
        const int W = im.W, H = im.H;
        const int ncols = (W - px + 1) >> 1;
        const int uy = u / ncols, ux = u - uy * ncols;
        const int x = 2 * ux + px, y = 2 * uy + py;
        const uint16_t *lab = im.lab[0];
        const int p = y * W + x;
        const int k = lab[p];
        int cand[4];
        const int nc = unit_candidates(lab, W, H, x, y, k, cand);
        if (nc > 0) {
            const int j = bin_at(im, p);
            // Prop. 2 sums G_x = sum_{i in K_p} b_{N_i}(x) as a weighted count
            // over the 5x5 window: w(p,q) = #{i in image: |i-p|,|i-q| <= 1}
            int Gk = 0, Gc[4] = {0, 0, 0, 0}, Kp = 0;
            if (im.patch != 0 && im.gnum != 0) {
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
                    if (wy[dy] == 0) continue;
                    const uint16_t *row = lab + (y + dy - 2) * W + (x - 2);
#pragma unroll
                    for (int dx = 0; dx < 5; ++dx) {
                        const int w = wx[dx] * wy[dy];
                        if (w == 0) continue;
                        const int l = row[dx];
                        if (l == k) Gk += w;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (c < nc && l == cand[c]) Gc[c] += w;
                    }
                }
            }
            const int64_t gd81 = 81ll * im.gden, gn = im.gnum;
            int best = cand[0];
            int64_t a_b = im.hist[hidx(im, best, j)], s_b = im.size[best];
            int G_b = Gc[0];
            for (int c = 1; c < nc; ++c) {
                const int n = cand[c];
                const int64_t a = im.hist[hidx(im, n, j)], sz = im.size[n];
                const int64_t diff = gd81 * (a * s_b - a_b * sz) + gn * (int64_t)(Gc[c] - G_b) * sz * s_b;
                if (diff > 0) {
                    best = n;
                    a_b = a;
                    s_b = sz;
                    G_b = Gc[c];
                }
            }
            const int64_t a_k = im.hist[hidx(im, k, j)], s_k = im.size[k];
            const int64_t gain =
                gd81 * (a_b * (s_k - 1) - (a_k - 1) * s_b) + gn * (int64_t)(G_b + Kp - Gk) * s_b * (s_k - 1);
            if (gain > 0) {
                has = true;
                w0 = (uint32_t)p;
                w1 = ((uint32_t)k << 16) | (uint32_t)best;
            }
        }
    }
    append_moves_warp(im, s, has, w0, w1, lane, err);
}

// ---------------------------------------------------------------------------
// block phase, small blocks: one thread per block (at most 16 pixels)
// ---------------------------------------------------------------------------

constexpr int kSmallMax = 16;

__device__ void op_block_phase_thread(const DevImage &im, int level, int phase, int units, int s, int u, int lane,
                                      int32_t *err)
{
    bool has = false;
    uint32_t w0 = 0, w1 = 0;
    if (u < units) {
        const int px = phase & 1, py = phase >> 1;
        const int nx = im.nbx[level], ny = im.nby[level];
        const int ncols = (nx - px + 1) >> 1;
        const int uy = u / ncols, ux = u - uy * ncols;
        const int bx = 2 * ux + px, by = 2 * uy + py;
        const uint16_t *lab = im.lab[level];
        const int k = lab[by * nx + bx];
        int cand[4];
        const int nc = unit_candidates(lab, nx, ny, bx, by, k, cand);
        if (nc > 0) {
            const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
            const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
            const int bw = x1 - x0, m = bw * (y1 - y0);
            int jj[kSmallMax];
#pragma unroll
            for (int t = 0; t < kSmallMax; ++t) {
                jj[t] = -1;
                if (t < m) {
                    const int dy = t / bw;
                    jj[t] = bin_at(im, (y0 + dy) * im.W + x0 + (t - dy * bw));
                }
            }
            int64_t S[4] = {0, 0, 0, 0}, S_st = 0;
            int64_t sz[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) sz[c] = c < nc ? im.size[cand[c]] : 1;
            const int64_t s_k = im.size[k], s_rest = s_k - m;
            // S(A, L) = sum over the distinct bins j of L of min(A[j]*|L|, L_j*|A|)
#pragma unroll
            for (int t = 0; t < kSmallMax; ++t) {
                if (t >= m) break;
                const int j = jj[t];
                bool first = true;
                int Lj = 0;
#pragma unroll
                for (int q = 0; q < kSmallMax; ++q) {
                    if (q < t && jj[q] == j) first = false;
                    if (q >= t && jj[q] == j) ++Lj;
                }
                if (!first) continue;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c < nc) S[c] += min((int64_t)im.hist[hidx(im, cand[c], j)] * m, (int64_t)Lj * sz[c]);
                S_st += min((int64_t)(im.hist[hidx(im, k, j)] - Lj) * m, (int64_t)Lj * s_rest);
            }
            int bi = 0;
#pragma unroll
            for (int c = 1; c < 4; ++c)
                if (c < nc && S[c] * sz[bi] > S[bi] * sz[c]) bi = c;
            if (S[bi] * s_rest > S_st * sz[bi]) {
                has = true;
                w0 = (uint32_t)(by * nx + bx);
                w1 = ((uint32_t)k << 16) | (uint32_t)cand[bi];
            }
        }
    }
    append_moves_warp(im, s, has, w0, w1, lane, err);
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

__device__ void op_block_phase_warp(const DevImage &im, int level, int phase, int units, int s, int u, int lane,
                                    int32_t *wsh, int max_nbins, int32_t *err)
{
    if (u >= units) return;
    const int px = phase & 1, py = phase >> 1;
    const int nx = im.nbx[level], ny = im.nby[level];
    const int ncols = (nx - px + 1) >> 1;
    const int uy = u / ncols, ux = u - uy * ncols;
    const int bx = 2 * ux + px, by = 2 * uy + py;
    const uint16_t *lab = im.lab[level];
    const int k = lab[by * nx + bx];
    int cand[4];
    const int nc = unit_candidates(lab, nx, ny, bx, by, k, cand);
    if (nc == 0) return;
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    const int bw = x1 - x0, m = bw * (y1 - y0);
    // the list lives past the largest histogram of the context, so that it
    // never overlaps histogram entries another image's blocks rely on being 0
    int32_t *ndist = wsh;
    int32_t *hsh = wsh + kScratchHeader;
    uint16_t *lst = (uint16_t *)(hsh + max_nbins);
    // sparse histogram of the block: counts in shared memory, distinct bins listed
    for (int base = 0; base < m; base += 32) {
        const int t = base + lane;
        const bool act = t < m;
        int j = -1;
        if (act) {
            const int dy = t / bw;
            j = bin_at(im, (y0 + dy) * im.W + x0 + (t - dy * bw));
        }
        const unsigned peers = __match_any_sync(0xffffffffu, j);
        if (act && lane == __ffs(peers) - 1) {
            const int old = atomicAdd(&hsh[j], __popc(peers));
            if (old == 0) lst[atomicAdd(ndist, 1)] = (uint16_t)j;
        }
    }
    __syncwarp();
    const int nd = *(volatile int32_t *)ndist;
    int64_t sz[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sz[c] = c < nc ? im.size[cand[c]] : 1;
    const int64_t s_k = im.size[k], s_rest = s_k - m;
    int64_t S[4] = {0, 0, 0, 0}, S_st = 0;
    for (int t = lane; t < nd; t += 32) {
        const int j = lst[t];
        const int Lj = hsh[j];
        hsh[j] = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < nc) S[c] += min((int64_t)im.hist[hidx(im, cand[c], j)] * m, (int64_t)Lj * sz[c]);
        S_st += min((int64_t)(im.hist[hidx(im, k, j)] - Lj) * m, (int64_t)Lj * s_rest);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) S[c] = warp_sum64(S[c]);
    S_st = warp_sum64(S_st);
    __syncwarp();
    if (lane == 0) {
        *ndist = 0;
        int bi = 0;
        for (int c = 1; c < nc; ++c)
            if (S[c] * sz[bi] > S[bi] * sz[c]) bi = c;
        if (S[bi] * s_rest > S_st * sz[bi])
            append_move_single(im, s, (uint32_t)(by * nx + bx), ((uint32_t)k << 16) | (uint32_t)cand[bi], err);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// descent, output
// ---------------------------------------------------------------------------

// level `level` -> level-1; the finer grid splits each block 2x2
__device__ void op_descend(const DevImage &im, int level, int64_t c)
{
    const int t = level - 1;
    if (t >= 1) {
        const int nx = im.nbx[t];
        if (c >= (int64_t)nx * im.nby[t]) return;
        const int cy = (int)(c / nx), cx = (int)(c - (int64_t)cy * nx);
        im.lab[t][c] = im.lab[level][(cy >> 1) * im.nbx[level] + (cx >> 1)];
    } else {
        const int W = im.W;
        if (c >= (int64_t)W * im.H) return;
        const int y = (int)(c / W), x = (int)(c - (int64_t)y * W);
        const int n1x = im.nbx[1], n1y = im.nby[1];
        // block b holds x iff floor(b*W/n) <= x < floor((b+1)*W/n)
        const int bx = (int)(((int64_t)(x + 1) * n1x - 1) / W);
        const int by = (int)(((int64_t)(y + 1) * n1y - 1) / im.H);
        im.lab[0][c] = im.lab[1][by * n1x + bx];
    }
}

__device__ void op_output(const DevImage &im, int64_t c)
{
    if (c < (int64_t)im.W * im.H) im.out[c] = im.lab[0][c];
}

// ---------------------------------------------------------------------------
// apply slot
// ---------------------------------------------------------------------------

__device__ __forceinline__ void move_hist(const DevImage &im, int k, int n, int j, int cnt)
{
    atomicSub(&im.hist[hidx(im, k, j)], cnt);
    atomicAdd(&im.hist[hidx(im, n, j)], cnt);
}

__device__ void apply_pixel(const DevImage &im, int m)
{
    const uint32_t p = im.moves[2 * m], w = im.moves[2 * m + 1];
    const int k = (int)(w >> 16), n = (int)(w & 0xFFFFu);
    const int j = bin_at(im, (int)p);
    im.lab[0][p] = (uint16_t)n;
    move_hist(im, k, n, j, 1);
    atomicSub(&im.size[k], 1);
    atomicAdd(&im.size[n], 1);
}

__device__ void apply_block_thread(const DevImage &im, int level, int m)
{
    const uint32_t u = im.moves[2 * m], w = im.moves[2 * m + 1];
    const int k = (int)(w >> 16), n = (int)(w & 0xFFFFu);
    const int nx = im.nbx[level];
    const int by = (int)(u / (uint32_t)nx), bx = (int)(u - (uint32_t)by * nx);
    im.lab[level][u] = (uint16_t)n;
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) move_hist(im, k, n, bin_at(im, y * im.W + x), 1);
    const int area = (x1 - x0) * (y1 - y0);
    atomicSub(&im.size[k], area);
    atomicAdd(&im.size[n], area);
}

__device__ void apply_block_warp(const DevImage &im, int level, int m, int lane)
{
    const uint32_t u = im.moves[2 * m], w = im.moves[2 * m + 1];
    const int k = (int)(w >> 16), n = (int)(w & 0xFFFFu);
    const int nx = im.nbx[level];
    const int by = (int)(u / (uint32_t)nx), bx = (int)(u - (uint32_t)by * nx);
    const int x0 = im.xe[level][bx], x1 = im.xe[level][bx + 1];
    const int y0 = im.ye[level][by], y1 = im.ye[level][by + 1];
    const int bw = x1 - x0, area = bw * (y1 - y0);
    for (int base = 0; base < area; base += 32) {
        const int t = base + lane;
        const bool act = t < area;
        int j = -1;
        if (act) {
            const int dy = t / bw;
            j = bin_at(im, (y0 + dy) * im.W + x0 + (t - dy * bw));
        }
        const unsigned peers = __match_any_sync(0xffffffffu, j);
        if (act && lane == __ffs(peers) - 1) move_hist(im, k, n, j, __popc(peers));
    }
    if (lane == 0) {
        im.lab[level][u] = (uint16_t)n;
        atomicSub(&im.size[k], area);
        atomicAdd(&im.size[n], area);
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(512) seeds_persistent(const DevImage *__restrict__ imgs, Schedule S,
                                                        GridBarrier *bar, int32_t *err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps_blk = blockDim.x >> 5;

    // per-warp scratch sized for the largest histogram of the context
    const int wbytes = warp_scratch_bytes(S.max_nbins);
    int32_t *wsh = (int32_t *)(smem + (size_t)warp * wbytes);
    for (int i = lane; i < wbytes / 4; i += 32) wsh[i] = 0;
    __syncwarp();

    const int64_t gwarp = (int64_t)blockIdx.x * nwarps_blk + warp;
    const int64_t nwarps = (int64_t)gridDim.x * nwarps_blk;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;

    const bool tracer = S.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
    if (tracer) S.trace[0] = global_ns();
    for (int s = 0; s < S.nsteps; ++s) {
        const int e0 = S.step_first[s], e1 = S.step_first[s + 1];
        // the other move counter of every image in this step was last read
        // by the previous apply slot; clear it for the next step
        if (blockIdx.x == 0)
            for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) imgs[S.ent[e].img].cnt[(s + 1) & 1] = 0;

        // ---- evaluate slot
        const int64_t total = S.step_vt[s];
        for (int64_t base = gwarp * 32; base < total; base += nwarps * 32) {
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
            const int64_t off = base - E.vt_begin;
            switch (E.op) {
            case OP_INIT:
                op_init(im, (int)(off >> 5), lane, wsh + kScratchHeader);
                break;
            case OP_PHASE:
                if (E.level == 0)
                    op_pixel_phase(im, E.phase, E.units, s, (int)(off + lane), lane, err);
                else if (E.group == 1)
                    op_block_phase_thread(im, E.level, E.phase, E.units, s, (int)(off + lane), lane, err);
                else
                    op_block_phase_warp(im, E.level, E.phase, E.units, s, (int)(off >> 5), lane, wsh, S.max_nbins,
                                        err);
                break;
            case OP_DESCEND:
                op_descend(im, E.level, off + lane);
                break;
            case OP_OUTPUT:
                op_output(im, off + lane);
                break;
            default:
                break;
            }
        }
        const bool last = s + 1 == S.nsteps;
        if (!S.step_apply[s]) {
            if (!last && !grid_sync(bar, err)) return;
            if (tracer) S.trace[1 + 2 * s] = S.trace[2 + 2 * s] = global_ns();
            continue;
        }
        if (!grid_sync(bar, err)) return;
        if (tracer) S.trace[1 + 2 * s] = global_ns();

        // ---- apply slot
        for (int e = e0; e < e1; ++e) {
            const StepEntry E = S.ent[e];
            if (E.op != OP_PHASE) continue;
            const DevImage &im = imgs[E.img];
            int count = ld_relaxed_i32(&im.cnt[s & 1]);
            if (count > im.moves_cap) {
                if (gtid == 0) atomicOr(err, DERR_BOUNDS);
                count = im.moves_cap;
            }
            if (E.level > 0 && E.group == 32) {
                for (int64_t m = gwarp; m < count; m += nwarps) apply_block_warp(im, E.level, (int)m, lane);
            } else if (E.level > 0) {
                for (int64_t m = gtid; m < count; m += nthreads) apply_block_thread(im, E.level, (int)m);
            } else {
                for (int64_t m = gtid; m < count; m += nthreads) apply_pixel(im, (int)m);
            }
        }
        if (!last && !grid_sync(bar, err)) return;
        if (tracer) S.trace[2 + 2 * s] = global_ns();
    }
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

// recount an image's histograms from the labels of one level (test hook)
__global__ void recount_kernel(const DevImage *imgs, int img, int level, int64_t npix, int phase_zero)
{
    const DevImage &im = imgs[img];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (phase_zero) {
        const int64_t nh = (int64_t)im.K * im.nbins;
        for (int64_t t = i; t < nh; t += (int64_t)gridDim.x * blockDim.x) im.hist[t] = 0;
        for (int64_t t = i; t < im.K; t += (int64_t)gridDim.x * blockDim.x) im.size[t] = 0;
        return;
    }
    if (i >= npix) return;
    const int y = (int)(i / im.W), x = (int)(i - (int64_t)y * im.W);
    int k;
    if (level == 0) {
        k = im.lab[0][i];
    } else {
        const int nx = im.nbx[level], ny = im.nby[level];
        const int bx = (int)(((int64_t)(x + 1) * nx - 1) / im.W);
        const int by = (int)(((int64_t)(y + 1) * ny - 1) / im.H);
        k = im.lab[level][by * nx + bx];
    }
    atomicAdd(&im.hist[hidx(im, k, bin_at(im, (int)i))], 1);
    atomicAdd(&im.size[k], 1);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

cudaError_t launch_set_io(DevImage *d_imgs, const IoChunk &chunk, cudaStream_t s)
{
    set_io_kernel<<<1, kIoChunk, 0, s>>>(d_imgs, chunk);
    return cudaGetLastError();
}

cudaError_t prepare_persistent(size_t smem)
{
    return cudaFuncSetAttribute(seeds_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t persistent_max_blocks_per_sm(int threads, size_t smem, int *n)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, seeds_persistent, threads, smem);
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

}  // namespace seeds

// ===========================================================================
// One image with no allocation at all: every byte of device state lives in a
// file-scope static device array.  For callers that may not allocate device
// memory (see seeds_run_static in seeds.h).
// ===========================================================================

#include <mutex>

namespace seeds {

static __device__ __align__(256) unsigned char g_static_scratch[SEEDS_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
unsigned char *g_static_addr[kStaticMaxDevices] = {};

// Host address stand-ins are not device addresses: ask the runtime, once per
// device, with that device current.
cudaError_t static_scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
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
    int32_t *apply;
    unsigned char *zero_begin;  // barrier, counters, error word
    int32_t zero_bytes;
    int32_t maxarea[kMaxLevels + 1];
    int32_t small_area;
    DevImage *img_out;
};

// Lays out one image inside the scratch: the image record, the block edge
// tables of every level, and the op schedule (one op per step); clears the
// barrier, the move counters and the error word.
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
    int s = 0, ne = 0;
    auto emit = [&](int kind, int level, int phase, int64_t units, int group) {
        S.first[s] = ne;
        const int64_t count = (units * group + 31) / 32 * 32;
        S.vt[s] = count;
        S.apply[s] = 0;
        if (count > 0) {
            StepEntry e;
            e.img = 0;
            e.op = kind;
            e.level = level;
            e.phase = phase;
            e.vt_begin = 0;
            e.units = (int32_t)units;
            e.group = group;
            S.ent[ne++] = e;
            S.apply[s] = kind == OP_PHASE;
        }
        ++s;
    };
    auto phase_units = [&](int l, int ph) {
        return (int64_t)((im.nbx[l] - (ph & 1) + 1) >> 1) * ((im.nby[l] - (ph >> 1) + 1) >> 1);
    };
    emit(OP_INIT, 0, 0, im.K, 32);
    for (int l = im.L; l >= 1; --l) {
        const int group = S.maxarea[l] > S.small_area ? 32 : 1;
        for (int it = 0; it < im.iters; ++it)
            for (int ph = 0; ph < 4; ++ph) emit(OP_PHASE, l, ph, phase_units(l, ph), group);
        emit(OP_DESCEND, l, 0, l - 1 >= 1 ? (int64_t)im.nbx[l - 1] * im.nby[l - 1] : (int64_t)im.W * im.H, 1);
    }
    for (int it = 0; it < im.iters; ++it)
        for (int ph = 0; ph < 4; ++ph) emit(OP_PHASE, 0, ph, phase_units(0, ph), 1);
    emit(OP_OUTPUT, 0, 0, (int64_t)im.W * im.H, 1);
    S.first[s] = ne;
}

__global__ void static_status_kernel(const int32_t *err, int32_t *status) { *status = *err; }

}  // namespace seeds

using namespace seeds;

extern "C" int seeds_run_static(const seeds_params *p, const uint8_t *d_rgb, int64_t row_stride_bytes,
                                int32_t *d_labels_out, int32_t *d_status, void *stream)
{
    // ---- parameters and grid (Sec. 5.1), arithmetic only
    if (!p || !d_rgb || !d_labels_out) return SEEDS_ERR_INVALID;
    if (p->width < 1 || p->height < 1 || p->width > 32768 || p->height > 32768) return SEEDS_ERR_INVALID;
    const int64_t N = (int64_t)p->width * p->height;
    if (N > 0x7fffffffLL || row_stride_bytes < 3 * (int64_t)p->width) return SEEDS_ERR_INVALID;
    if (p->num_superpixels < 1 || p->block_levels < 0 || p->block_levels > kMaxLevels) return SEEDS_ERR_INVALID;
    if (p->bins_per_channel < 1 || p->bins_per_channel > 16) return SEEDS_ERR_INVALID;
    if (p->iters_per_level < 1 || p->iters_per_level > 1000) return SEEDS_ERR_INVALID;
    if (p->patch != 0 && p->patch != 3) return SEEDS_ERR_INVALID;
    if (p->gamma_num < 0 || p->gamma_num > 1024 || p->gamma_den < 1 || p->gamma_den > 1024) return SEEDS_ERR_INVALID;
    const double Kd = p->num_superpixels, Wd = p->width, Hd = p->height;
    long long gx = std::llround(std::sqrt(Kd * Wd / Hd));
    if (gx < 1) gx = 1;
    long long gy = std::llround(Kd / (double)gx);
    if (gy < 1) gy = 1;
    if (gx * gy > 65535) return SEEDS_ERR_INVALID;
    const int L = p->block_levels;
    if ((gx << L) > p->width || (gy << L) > p->height) return SEEDS_ERR_GEOMETRY;
    const int B = p->bins_per_channel, nbins = B * B * B, K = (int)(gx * gy);

    StaticSetup S;
    std::memset(&S, 0, sizeof(S));
    DevImage &d = S.img;
    d.W = p->width;
    d.H = p->height;
    d.K = K;
    d.gx = (int)gx;
    d.gy = (int)gy;
    d.L = L;
    d.iters = p->iters_per_level;
    d.B = B;
    d.nbins = nbins;
    d.patch = p->patch;
    d.gnum = p->gamma_num;
    d.gden = p->gamma_den;
    d.bins16 = nbins > 256;
    d.hist_jmajor = 0;
    d.nbx[0] = p->width;
    d.nby[0] = p->height;
    int amax = 1;
    for (int l = 1; l <= L; ++l) {
        d.nbx[l] = (int)(gx << (L - l + 1));
        d.nby[l] = (int)(gy << (L - l + 1));
        const int mw = (p->width + d.nbx[l] - 1) / d.nbx[l], mh = (p->height + d.nby[l] - 1) / d.nby[l];
        S.maxarea[l] = mw * mh;
        amax = std::max(amax, mw * mh);
    }
    const __int128 N2 = (__int128)N * N, lim = ((__int128)1) << 63;
    if ((__int128)amax * N2 >= lim || (__int128)(81 * p->gamma_den + 90 * p->gamma_num) * N2 >= lim)
        return SEEDS_ERR_INT64;
    S.small_area = 16;
    const int nops = 1 + (L + 1) * 4 * p->iters_per_level + L + 1;
    const int moves_cap = (int)(((int64_t)(p->width + 1) / 2) * ((p->height + 1) / 2));

    // ---- layout inside the scratch
    size_t off = 0;
    const size_t o_img = off;
    off = sal(off + sizeof(DevImage));
    const size_t o_zero = off;  // barrier | 2 counters | error word
    const size_t o_bar = off, o_cnt = off + 16, o_err = off + 32;
    off = sal(off + 64);
    const size_t o_ent = off;
    off = sal(off + sizeof(StepEntry) * (size_t)nops);
    const size_t o_first = off;
    off = sal(off + 4 * (size_t)(nops + 1));
    const size_t o_vt = off;
    off = sal(off + 8 * (size_t)nops);
    const size_t o_apply = off;
    off = sal(off + 4 * (size_t)nops);
    size_t o_xe[kMaxLevels + 1] = {}, o_ye[kMaxLevels + 1] = {}, o_lab[kMaxLevels + 1] = {};
    for (int l = 1; l <= L; ++l) {
        o_xe[l] = off;
        off = sal(off + 4 * (size_t)(d.nbx[l] + 1));
        o_ye[l] = off;
        off = sal(off + 4 * (size_t)(d.nby[l] + 1));
    }
    const size_t o_bins = off;
    off = sal(off + (size_t)N * (d.bins16 ? 2 : 1));
    for (int l = 0; l <= L; ++l) {
        o_lab[l] = off;
        off = sal(off + 2 * (size_t)d.nbx[l] * d.nby[l]);
    }
    const size_t o_hist = off;
    off = sal(off + 4 * (size_t)K * nbins);
    const size_t o_size = off;
    off = sal(off + 4 * (size_t)K);
    const size_t o_moves = off;
    off = sal(off + 8 * (size_t)moves_cap);
    if (off > (size_t)SEEDS_STATIC_SCRATCH_BYTES) return SEEDS_ERR_STATIC_SIZE;

    // ---- the scratch's device address on the current device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SEEDS_ERR_CUDA;
    unsigned char *base = nullptr;
    if (static_scratch_address(dev, &base) != cudaSuccess) return SEEDS_ERR_CUDA;

    for (int l = 0; l <= L; ++l) d.lab[l] = (uint16_t *)(base + o_lab[l]);
    for (int l = 1; l <= L; ++l) {
        d.xe[l] = (const int32_t *)(base + o_xe[l]);
        d.ye[l] = (const int32_t *)(base + o_ye[l]);
    }
    d.bins = base + o_bins;
    d.hist = (int32_t *)(base + o_hist);
    d.size = (int32_t *)(base + o_size);
    d.moves = (uint32_t *)(base + o_moves);
    d.moves_cap = moves_cap;
    d.cnt = (int32_t *)(base + o_cnt);
    d.rgb = d_rgb;
    d.stride = row_stride_bytes;
    d.out = d_labels_out;
    S.ent = (StepEntry *)(base + o_ent);
    S.first = (int32_t *)(base + o_first);
    S.vt = (int64_t *)(base + o_vt);
    S.apply = (int32_t *)(base + o_apply);
    S.zero_begin = base + o_zero;
    S.zero_bytes = 64;
    S.img_out = (DevImage *)(base + o_img);

    // ---- launch configuration of the persistent kernel (as a context would)
    const int threads = 256;
    const size_t smem = (size_t)(threads / 32) * warp_scratch_bytes(nbins);
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SEEDS_ERR_CUDA;
    if (prepare_persistent(smem) != cudaSuccess) return SEEDS_ERR_CUDA;
    if (persistent_max_blocks_per_sm(threads, smem, &per_sm) != cudaSuccess || per_sm < 1) return SEEDS_ERR_CUDA;

    cudaStream_t s = (cudaStream_t)stream;
    static_setup_kernel<<<8, 256, 0, s>>>(S);
    if (cudaGetLastError() != cudaSuccess) return SEEDS_ERR_CUDA;
    Schedule sch;
    sch.ent = S.ent;
    sch.step_first = S.first;
    sch.step_vt = S.vt;
    sch.step_apply = S.apply;
    sch.nsteps = nops;
    sch.max_nbins = nbins;
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
