// seeds_host.h -- host-side helpers shared by the context runtime and the
// serving runtime: parameter validation, grid geometry, the device layout of
// one image's state, and its device record.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "seeds.h"
#include "seeds_device.cuh"

namespace seeds {
namespace host {

struct Op {
    int kind, level, phase;
};

// The heap-free description of one image: its parameters, the grid and
// block levels derived from them, and the byte offsets of its device state
// inside one allocation (or inside the static scratch of seeds_run_static).
struct ImageCore {
    seeds_params p{};
    int gx = 0, gy = 0, K = 0, L = 0, B = 0, nbins = 0;
    int64_t N = 0;
    int nbx[kMaxLevels + 1] = {}, nby[kMaxLevels + 1] = {};
    int maxarea[kMaxLevels + 1] = {};
    int nops = 0;
    int units_cap = 0;
    // byte offsets of the state, from the image's base address
    size_t off_bins = 0, off_lab[kMaxLevels + 1][2] = {}, off_xe[kMaxLevels + 1] = {}, off_ye[kMaxLevels + 1] = {};
    size_t off_hist[2] = {}, off_size[2] = {}, off_dec[2] = {}, off_msum[2] = {}, off_edges = 0, bytes = 0;
};

// An image of a context or of the server: the core plus its block edge
// tables (uploaded once) and its op list.
struct ImageHost : ImageCore {
    std::vector<int32_t> xe[kMaxLevels + 1], ye[kMaxLevels + 1];
    std::vector<Op> ops;  // full list, output op last
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

inline int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return SEEDS_OK;
    if (e == cudaErrorMemoryAllocation) return SEEDS_ERR_NO_MEMORY;
    return SEEDS_ERR_CUDA;
}

// Validate one image's parameters and derive its grid (gx, gy) and block
// levels: gx = max(1, round(sqrt(K*W/H))), gy = max(1, round(K/gx)), level-l
// edges floor(i*W/(gx*2^(L-l+1))) (Sec. 5.1).  Checks the int64 bound of the
// exact compares and lays out the image's device state.  Allocates nothing:
// the allocation-free entry point runs it as it is.  gx_out / gy_out receive
// the grid as soon as it is known (also when the levels do not fit).
inline int derive_core(const seeds_params *p, ImageCore *g, int32_t *gx_out, int32_t *gy_out)
{
    if (!p) return SEEDS_ERR_INVALID;
    if (p->width < 1 || p->height < 1 || p->width > 32768 || p->height > 32768) return SEEDS_ERR_INVALID;
    const int64_t N = (int64_t)p->width * p->height;
    if (N > 0x7fffffffLL) return SEEDS_ERR_INVALID;
    if (p->num_superpixels < 1) return SEEDS_ERR_INVALID;
    if (p->block_levels < 0 || p->block_levels > kMaxLevels) return SEEDS_ERR_INVALID;
    if (p->bins_per_channel < 1 || p->bins_per_channel > 16) return SEEDS_ERR_INVALID;
    if (p->iters_per_level < 0 || p->iters_per_level > 1000) return SEEDS_ERR_INVALID;
    if (p->iters_per_level == 0 && p->means_iters == 0) return SEEDS_ERR_INVALID;  // SPM alone needs means
    if (p->patch != 0 && p->patch != 3) return SEEDS_ERR_INVALID;
    if (p->color_space != 0 && p->color_space != 1) return SEEDS_ERR_INVALID;
    if (p->means_iters < 0 || p->means_iters > 1000) return SEEDS_ERR_INVALID;
    if (p->compactness < 0 || p->compactness > 1024) return SEEDS_ERR_INVALID;
    if (p->edge_threshold < 0 || p->edge_threshold > 765) return SEEDS_ERR_INVALID;
    if (p->compact_prior < 0 || p->compact_prior > 1024) return SEEDS_ERR_INVALID;
    if (p->gamma_num < 0 || p->gamma_num > 1024 || p->gamma_den < 1 || p->gamma_den > 1024) return SEEDS_ERR_INVALID;
    const double Kd = p->num_superpixels, Wd = p->width, Hd = p->height;
    long long gx = std::llround(std::sqrt(Kd * Wd / Hd));
    if (gx < 1) gx = 1;
    long long gy = std::llround(Kd / (double)gx);
    if (gy < 1) gy = 1;
    if (gx * gy > 65535) return SEEDS_ERR_INVALID;  // labels are 16-bit
    if (gx_out) *gx_out = (int32_t)gx;
    if (gy_out) *gy_out = (int32_t)gy;
    const int L = p->block_levels;
    if ((gx << L) > p->width || (gy << L) > p->height) return SEEDS_ERR_GEOMETRY;

    ImageCore local;
    ImageCore &h = g ? *g : local;
    h.p = *p;
    h.gx = (int)gx;
    h.gy = (int)gy;
    h.K = (int)(gx * gy);
    h.L = L;
    h.B = p->bins_per_channel;
    h.nbins = h.B * h.B * h.B;
    h.N = N;
    h.nbx[0] = p->width;
    h.nby[0] = p->height;
    h.maxarea[0] = 1;
    int amax = 1;
    for (int l = 1; l <= L; ++l) {
        h.nbx[l] = (int)(gx << (L - l + 1));
        h.nby[l] = (int)(gy << (L - l + 1));
        // floor edges floor(i*W/n) give widths floor(W/n) and ceil(W/n); the
        // widths add up to W, so ceil(W/n) occurs whenever n does not divide
        // W: the widest block spans ceil(W/n) columns, the tallest
        // ceil(H/n) rows, and blocks form a tensor product
        const int mw = (p->width + h.nbx[l] - 1) / h.nbx[l], mh = (p->height + h.nby[l] - 1) / h.nby[l];
        h.maxarea[l] = mw * mh;
        amax = std::max(amax, mw * mh);
    }
    // exact int64 compares: block products reach |L|max*N^2, pixel products
    // (81*gamma_den + 90*gamma_num)*N^2
    const __int128 N2 = (__int128)N * N;
    const __int128 lim = ((__int128)1) << 63;
    if ((__int128)amax * N2 >= lim) return SEEDS_ERR_INT64;
    if ((__int128)(81 * p->gamma_den + 90 * p->gamma_num) * N2 >= lim) return SEEDS_ERR_INT64;
    h.nops = num_ops(L, p->iters_per_level, p->means_iters);
    h.units_cap = (int)(((int64_t)(p->width + 1) / 2) * ((p->height + 1) / 2));

    // device layout: bins, then two buffers of every label grid, the block
    // edge tables, and two buffers of every histogram, size vector and
    // decision array
    size_t off = 0;
    h.off_bins = off;
    off = align_up(off + (size_t)N * (h.nbins > 256 ? 2 : 1));
    for (int l = 0; l <= L; ++l)
        for (int q = 0; q < 2; ++q) {
            h.off_lab[l][q] = off;
            off = align_up(off + (size_t)h.nbx[l] * h.nby[l] * 2);
        }
    for (int l = 1; l <= L; ++l) {
        h.off_xe[l] = off;
        off = align_up(off + (h.nbx[l] + 1) * 4);
        h.off_ye[l] = off;
        off = align_up(off + (h.nby[l] + 1) * 4);
    }
    for (int q = 0; q < 2; ++q) {
        h.off_hist[q] = off;
        off = align_up(off + (size_t)h.K * h.nbins * 4);
        h.off_size[q] = off;
        off = align_up(off + (size_t)h.K * 4);
        h.off_dec[q] = off;
        off = align_up(off + (size_t)h.units_cap * 4);
        h.off_msum[q] = off;  // per superpixel sums: means iterations, compactness prior
        if (p->means_iters > 0 || p->compact_prior > 0) off = align_up(off + (size_t)h.K * 5 * 8);
    }
    h.off_edges = off;  // the edge-snapping mask
    if (p->edge_threshold > 0) off = align_up(off + (size_t)N);
    h.bytes = off;
    return SEEDS_OK;
}

// derive_core plus the host copies of the block edge tables and the op list
// (the same one the kernels derive with op_at).
inline int derive(const seeds_params *p, ImageHost *g, int32_t *gx_out, int32_t *gy_out)
{
    ImageHost local;
    ImageHost &h = g ? *g : local;
    const int rc = derive_core(p, &h, gx_out, gy_out);
    if (rc || !g) return rc;
    for (int l = 1; l <= h.L; ++l) {
        h.xe[l].resize(h.nbx[l] + 1);
        h.ye[l].resize(h.nby[l] + 1);
        for (int i = 0; i <= h.nbx[l]; ++i) h.xe[l][i] = (int32_t)((int64_t)i * h.p.width / h.nbx[l]);
        for (int i = 0; i <= h.nby[l]; ++i) h.ye[l][i] = (int32_t)((int64_t)i * h.p.height / h.nby[l]);
    }
    h.ops.clear();
    for (int o = 0; o < h.nops; ++o) {
        const OpDesc d = op_at(h.L, h.p.iters_per_level, h.p.means_iters, o);
        h.ops.push_back({d.kind, d.level, d.phase});
    }
    return SEEDS_OK;
}


// The device record of an image whose state starts at `base` (laid out as
// derive() planned), with the given launch knobs and per-call pointers.
// The fields of an image's device record that its op list and step
// schedule depend on (size, grids, levels, iterations, launch knobs), with
// no device pointer: enough to plan a schedule on a host without a GPU.
inline DevImage plan_image(const ImageCore &h, const seeds_tuning &t)
{
    DevImage d;
    std::memset(&d, 0, sizeof(d));
    d.W = h.p.width;
    d.H = h.p.height;
    d.K = h.K;
    d.gx = h.gx;
    d.gy = h.gy;
    d.L = h.L;
    d.iters = h.p.iters_per_level;
    d.means_iters = h.p.means_iters;
    d.small_area = t.small_block_area;
    d.tile_uy = t.pixel_tile_rows == 2 ? 2 : kTileUY;
    for (int l = 0; l <= h.L; ++l) {
        d.nbx[l] = h.nbx[l];
        d.nby[l] = h.nby[l];
        d.maxarea[l] = h.maxarea[l];
    }
    return d;
}

inline DevImage make_dev_image(const ImageCore &h, unsigned char *base, const seeds_tuning &t, const IoEntry &io,
                               int32_t *err)
{
    DevImage d = plan_image(h, t);
    d.B = h.B;
    d.nbins = h.nbins;
    d.patch = h.p.patch;
    d.color = h.p.color_space;
    // SLIC's (m/S)^2 with S^2 = N/K
    d.means_w = (float)((int64_t)h.p.compactness * h.p.compactness * h.K) / (float)h.N;
    // the compactness prior: (compact_prior/16) * D * K / N, and gamma as a float
    d.prior = h.p.compact_prior > 0;
    d.compact_w = (float)((int64_t)h.p.compact_prior * 81 * h.K) / (float)((int64_t)16 * h.N);
    d.gamma_f = h.p.patch == 3 ? (float)h.p.gamma_num / (float)h.p.gamma_den : 0.0f;
    d.edge_tau = h.p.edge_threshold;
    d.edges = h.p.edge_threshold > 0 ? base + h.off_edges : nullptr;
    d.gnum = h.p.gamma_num;
    d.gden = h.p.gamma_den;
    d.bins16 = h.nbins > 256;
    d.hist_jmajor = t.hist_layout == 1;
    d.hist_sk = d.hist_jmajor ? 1 : h.nbins;
    d.hist_sj = d.hist_jmajor ? h.K : 1;
    for (int l = 0; l <= h.L; ++l) {
        for (int q = 0; q < 2; ++q) d.lab[l][q] = (uint16_t *)(base + h.off_lab[l][q]);
        if (l >= 1) {
            d.xe[l] = (const int32_t *)(base + h.off_xe[l]);
            d.ye[l] = (const int32_t *)(base + h.off_ye[l]);
        }
    }
    d.bins = base + h.off_bins;
    for (int q = 0; q < 2; ++q) {
        d.hist[q] = (int32_t *)(base + h.off_hist[q]);
        d.size[q] = (int32_t *)(base + h.off_size[q]);
        d.dec[q] = (uint32_t *)(base + h.off_dec[q]);
        d.msum[q] = h.p.means_iters > 0 || d.prior ? (unsigned long long *)(base + h.off_msum[q]) : nullptr;
    }
    d.units_cap = h.units_cap;
    d.err = err;
    d.rgb = io.rgb;
    d.stride = io.stride;
    d.out = io.out;
    return d;
}

// The autotuner's search: coordinate descent over the result-invariant
// launch knobs (threads per CTA, CTAs per SM, histogram layout, small-block
// area, tile rows, block tiles), one pass in that order, from `start`.  cost(t, &ms)
// times a setting (ms = +inf if it cannot run; a nonzero return aborts the
// search with that status); a value replaces the current one only if it is
// at least 2% faster, so timing noise does not move the setting.
template <class Cost>
inline int tune_search(const seeds_tuning &start, Cost cost, seeds_tuning *best)
{
    seeds_tuning cur = start;
    float cur_ms = 0.f;
    int rc = cost(cur, &cur_ms);
    const int threads[] = {128, 256, 512, 1024}, blocks[] = {0, 1, 2, 3}, layouts[] = {0, 1}, areas[] = {4, 9, 16},
              rows[] = {2, 4}, tiles[] = {0, 1, 2};
    for (int knob = 0; knob < 6 && !rc; ++knob) {
        const int *vals = knob == 0   ? threads
                          : knob == 1 ? blocks
                          : knob == 2 ? layouts
                          : knob == 3 ? areas
                          : knob == 4 ? rows
                                      : tiles;
        const int nv = knob == 0 ? 4 : knob == 1 ? 4 : knob == 2 ? 2 : knob == 3 ? 3 : knob == 4 ? 2 : 3;
        for (int v = 0; v < nv && !rc; ++v) {
            seeds_tuning t = cur;
            int *field = knob == 0   ? &t.threads_per_block
                         : knob == 1 ? &t.blocks_per_sm
                         : knob == 2 ? &t.hist_layout
                         : knob == 3 ? &t.small_block_area
                         : knob == 4 ? &t.pixel_tile_rows
                                     : &t.block_tiles;
            if (*field == vals[v]) continue;
            *field = vals[v];
            float ms = 0.f;
            rc = cost(t, &ms);
            if (!rc && ms < 0.98f * cur_ms) {
                cur = t;
                cur_ms = ms;
            }
        }
    }
    *best = cur;
    return rc;
}

// The step schedule of a set of images: image i runs its ops [b[i], e[i]),
// one op per step; pend[i] says that the moves of op b[i]-1 are still
// pending, so its first step catches them up.  Appends the entries of every
// step to `ent`, the index of each step's first entry to `first` (and one
// past the last step's), and each step's padded thread count to `vt`.  Each
// step is planned three times: with every replay fused, per-unit block
// entries and then block tiles, to measure it, then with the mode step_mode
// chooses for those sizes against split_below warps and tile_policy.
inline void build_steps(const std::vector<DevImage> &imgs, const std::vector<int> &b, const std::vector<int> &e,
                        const std::vector<char> &pend, int64_t split_below, int tile_policy, std::vector<StepEntry> &ent,
                        std::vector<int32_t> &first, std::vector<int64_t> &vt)
{
    const int n = (int)imgs.size();
    int nsteps = 0;
    for (int i = 0; i < n; ++i) nsteps = std::max(nsteps, e[i] - b[i]);
    StepEntry two[2];
    for (int s = 0; s < nsteps; ++s) {
        first.push_back((int32_t)ent.size());
        int64_t sized[2] = {0, 0};
        for (int pass = 0; pass < 3; ++pass) {
            int64_t v = 0;
            const int mode =
                pass == 0 ? 2 : pass == 1 ? 2 | kWideStep : step_mode(sized[0], sized[1], split_below, tile_policy);
            for (int i = 0; i < n; ++i) {
                const DevImage &im = imgs[i];
                const int o = b[i] + s;
                if (o >= e[i]) continue;
                const bool catchup =
                    s == 0 ? (o > 0 && pend[i]) : is_phase(op_at(im.L, im.iters, im.means_iters, o - 1).kind);
                const int m = emit_entries(im, i, o, catchup, mode, two, &v);
                if (pass == 2)
                    for (int q = 0; q < m; ++q) ent.push_back(two[q]);
            }
            if (pass < 2)
                sized[pass] = v;
            else
                vt.push_back(v);
        }
    }
    first.push_back((int32_t)ent.size());
}

}  // namespace host
}  // namespace seeds
