// seeds_runtime.cu -- host runtime behind the C ABI of include/seeds.h.
//
// Validates parameters and derives each image's grid geometry, lays out all
// device state of a context in one allocation, builds and caches the step
// schedules the persistent kernel walks, and issues the launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "seeds.h"
#include "seeds_device.cuh"
#include "seeds_host.h"

using namespace seeds;

using namespace seeds::host;

namespace {

struct DevSchedule {
    void *buf = nullptr;
    Schedule s{};
};

}  // namespace

struct seeds_ctx {
    int device = 0;
    int sm_count = 0;
    std::vector<ImageHost> img;
    std::vector<DevImage> h_imgs;
    std::vector<IoEntry> io;
    DevImage *d_imgs = nullptr;
    unsigned char *pool = nullptr;
    size_t pool_bytes = 0;
    std::vector<int> cur;      // per image: ops done in the current chain (state in buffer cur & 1)
    std::vector<int> pending;  // per image: op whose moves await catch-up, or -1
    GridBarrier *d_bar = nullptr;
    int32_t *d_err = nullptr;
    int32_t *d_steps = nullptr;  // steps run by the last anytime launch
    bool stopped_state = false;  // the last launch was an anytime run: no final state to output
    seeds_tuning tune{1024, 0, 0, 16, 4, 0};
    int grid = 0;
    size_t smem = 0;
    int max_nbins = 1;
    std::map<std::string, DevSchedule> schedules;
    cudaEvent_t done = nullptr;
    bool launched = false;
    bool profile = false, profiled = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    unsigned long long *d_trace = nullptr;  // step stamps while profiling
    int trace_cap = 0, traced_steps = 0;
    int64_t launches = 0;
    unsigned long long dbg_timeout_ns = 0;  // failure tests: barrier limit, withheld arrival
    int32_t dbg_withhold = 0;
    unsigned char *stage[2] = {};  // host-run staging: slot 0 (seeds_run_host), slot 1 (streams)
    size_t stage_bytes = 0;        // per slot
    std::vector<size_t> stage_rgb, stage_out;
    // seeds_run_host_stream: copy streams and the events that order them
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_entry = nullptr, ev_in[2] = {}, ev_k[2] = {}, ev_out[2] = {};
};

namespace {

enum { SCHED_ITERATE = 0, SCHED_FULL = 1, SCHED_OUTPUT = 2, SCHED_DEBUG = 3 };

void free_schedules(seeds_ctx *c)
{
    for (auto &kv : c->schedules) cudaFree(kv.second.buf);
    c->schedules.clear();
}

int configure_launch(seeds_ctx *c)
{
    const int threads = c->tune.threads_per_block;
    c->smem = (size_t)(threads / 32) * warp_scratch_bytes(c->max_nbins);
    int rc = from_cuda(prepare_persistent(c->smem));
    if (rc) return rc;
    int per_sm = 0;
    rc = from_cuda(persistent_max_blocks_per_sm(threads, c->smem, &per_sm));
    if (rc) return rc;
    if (per_sm < 1) return SEEDS_ERR_INVALID;
    if (c->tune.blocks_per_sm > 0) per_sm = std::min(per_sm, c->tune.blocks_per_sm);
    c->grid = per_sm * c->sm_count;
    return SEEDS_OK;
}

void fill_dev_images(seeds_ctx *c)
{
    c->h_imgs.resize(c->img.size());
    unsigned char *base = c->pool;
    for (size_t i = 0; i < c->img.size(); ++i) {
        c->h_imgs[i] = make_dev_image(c->img[i], base, c->tune, c->io[i], c->d_err);
        base += c->img[i].bytes;
    }
}

// per-image op ranges [b, e) for a schedule kind
void op_range(const ImageHost &h, int kind, int ob, int oe, int *b, int *e)
{
    const int n = (int)h.ops.size();
    switch (kind) {
    case SCHED_ITERATE:
        *b = 0;
        *e = n - 1;
        break;
    case SCHED_FULL:
        *b = 0;
        *e = n;
        break;
    case SCHED_OUTPUT:
        *b = n - 1;
        *e = n;
        break;
    default:
        *b = std::min(std::max(ob, 0), n - 1);
        *e = std::min(std::max(oe, *b), n - 1);
        break;
    }
}

// Build (or reuse) the schedule running ops [b_i, e_i) of every image i, one
// op per step; the first op of an image catches up the moves of the op
// before it when those are still pending from an earlier launch.
int get_schedule(seeds_ctx *c, int kind, int ob, int oe, const Schedule **out)
{
    const int n = (int)c->img.size();
    std::vector<int> b(n), e(n);
    std::string key = std::to_string(kind) + ":" + std::to_string(ob) + ":" + std::to_string(oe) + ":";
    int nsteps = 0;
    for (int i = 0; i < n; ++i) {
        op_range(c->img[i], kind, ob, oe, &b[i], &e[i]);
        nsteps = std::max(nsteps, e[i] - b[i]);
        key += (b[i] > 0 && c->pending[i] == b[i] - 1) ? '1' : '0';
    }
    auto it = c->schedules.find(key);
    if (it != c->schedules.end()) {
        *out = &it->second.s;
        return SEEDS_OK;
    }
    std::vector<StepEntry> ent;
    std::vector<int32_t> first;
    std::vector<int64_t> vt;
    std::vector<char> pend(n);
    for (int i = 0; i < n; ++i) pend[i] = b[i] > 0 && c->pending[i] == b[i] - 1;
    build_steps(c->h_imgs, b, e, pend, (int64_t)c->sm_count * 32, c->tune.block_tiles, ent, first, vt);
    if (ent.empty()) ent.push_back(StepEntry{});  // keep the buffer non-empty

    const size_t b_ent = align_up(ent.size() * sizeof(StepEntry));
    const size_t b_first = align_up(first.size() * sizeof(int32_t));
    const size_t b_vt = align_up(std::max<size_t>(1, vt.size()) * sizeof(int64_t));
    DevSchedule ds;
    int rc = from_cuda(cudaMalloc(&ds.buf, b_ent + b_first + b_vt));
    if (rc) return rc;
    unsigned char *p = (unsigned char *)ds.buf;
    std::vector<unsigned char> host(b_ent + b_first + b_vt, 0);
    std::memcpy(host.data(), ent.data(), ent.size() * sizeof(StepEntry));
    std::memcpy(host.data() + b_ent, first.data(), first.size() * sizeof(int32_t));
    if (!vt.empty()) std::memcpy(host.data() + b_ent + b_first, vt.data(), vt.size() * sizeof(int64_t));
    rc = from_cuda(cudaMemcpy(ds.buf, host.data(), host.size(), cudaMemcpyHostToDevice));
    if (rc) {
        cudaFree(ds.buf);
        return rc;
    }
    ds.s.ent = (const StepEntry *)p;
    ds.s.step_first = (const int32_t *)(p + b_ent);
    ds.s.step_vt = (const int64_t *)(p + b_ent + b_first);
    ds.s.nsteps = nsteps;
    ds.s.max_nbins = c->max_nbins;
    ds.s.trace = nullptr;
    ds.s.nimg = n;
    auto ins = c->schedules.emplace(key, ds);
    *out = &ins.first->second.s;
    return SEEDS_OK;
}

// push the per-call pointers of every image to the device records
int push_io(seeds_ctx *c, cudaStream_t s)
{
    const int n = (int)c->img.size();
    for (int f = 0; f < n; f += kIoChunk) {
        IoChunk ch;
        std::memset(&ch, 0, sizeof(ch));
        ch.first = f;
        ch.n = std::min(kIoChunk, n - f);
        for (int t = 0; t < ch.n; ++t) ch.e[t] = c->io[f + t];
        int rc = from_cuda(launch_set_io(c->d_imgs, ch, s));
        if (rc) return rc;
        ++c->launches;
    }
    return SEEDS_OK;
}

// Launch the schedule of `kind`; stop_steps / budget_ns > 0 make it an
// anytime run (full schedules only).
int launch(seeds_ctx *c, int kind, int ob, int oe, cudaStream_t s, int32_t stop_steps = 0, int64_t budget_ns = 0)
{
    const Schedule *sch = nullptr;
    int rc = get_schedule(c, kind, ob, oe, &sch);
    if (rc) return rc;
    rc = push_io(c, s);
    if (rc) return rc;
    if (sch->nsteps == 0) return SEEDS_OK;
    rc = from_cuda(cudaMemsetAsync(c->d_bar, 0, sizeof(GridBarrier), s));
    if (rc) return rc;
    Schedule run = *sch;
    run.trace = nullptr;
    const bool anytime = stop_steps > 0 || budget_ns > 0;
    run.stop_steps = stop_steps;
    run.budget_ns = (unsigned long long)budget_ns;
    run.steps_out = anytime ? c->d_steps : nullptr;
    run.timeout_ns = c->dbg_timeout_ns;
    run.withhold = c->dbg_withhold;
    if (c->profile) {
        rc = from_cuda(cudaEventRecord(c->ev0, s));
        if (rc) return rc;
        if (1 + run.nsteps <= c->trace_cap) {
            run.trace = c->d_trace;
            c->traced_steps = run.nsteps;
        } else {
            c->traced_steps = 0;
        }
    }
    rc = from_cuda(launch_persistent(c->d_imgs, run, c->d_bar, c->d_err, c->grid, c->tune.threads_per_block,
                                     c->smem, s));
    if (rc) return rc;
    ++c->launches;
    if (c->profile) {
        rc = from_cuda(cudaEventRecord(c->ev1, s));
        if (rc) return rc;
    }
    c->profiled = c->profile;
    // while the stream is being captured into a CUDA graph the completion
    // event keeps its last real record: the caller synchronises replays
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    rc = from_cuda(cudaStreamIsCapturing(s, &cap));
    if (!rc && cap == cudaStreamCaptureStatusNone) rc = from_cuda(cudaEventRecord(c->done, s));
    c->launched = true;
    // where every image's state now lives, and which moves await catch-up
    c->stopped_state = anytime;
    for (size_t i = 0; i < c->img.size(); ++i) {
        if (anytime) {  // the state is that of wherever the launch stopped
            c->cur[i] = 0;
            c->pending[i] = -1;
            continue;
        }
        int b = 0, e = 0;
        op_range(c->img[i], kind, ob, oe, &b, &e);
        if (e <= b) continue;
        c->cur[i] = e;
        c->pending[i] = is_phase(c->img[i].ops[e - 1].kind) ? e - 1 : -1;
    }
    return rc;
}

void destroy_ctx(seeds_ctx *c)
{
    if (!c) return;
    if (c->launched) cudaEventSynchronize(c->done);
    free_schedules(c);
    cudaFree(c->d_imgs);
    cudaFree(c->pool);
    cudaFree(c->d_bar);
    cudaFree(c->d_err);
    cudaFree(c->d_steps);
    cudaFree(c->stage[0]);
    cudaFree(c->stage[1]);
    if (c->s_in) {
        cudaStreamSynchronize(c->s_in);
        cudaStreamSynchronize(c->s_out);
        cudaStreamDestroy(c->s_in);
        cudaStreamDestroy(c->s_out);
    }
    for (cudaEvent_t e : {c->ev_entry, c->ev_in[0], c->ev_in[1], c->ev_k[0], c->ev_k[1], c->ev_out[0], c->ev_out[1]})
        if (e) cudaEventDestroy(e);
    cudaFree(c->d_trace);
    if (c->done) cudaEventDestroy(c->done);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

int create_ctx(const seeds_params *p, int32_t n, seeds_ctx **out)
{
    if (!p || !out || n < 1 || n > SEEDS_MAX_BATCH) return SEEDS_ERR_INVALID;
    *out = nullptr;
    seeds_ctx *c = new (std::nothrow) seeds_ctx;
    if (!c) return SEEDS_ERR_NO_MEMORY;
    c->img.resize(n);
    for (int i = 0; i < n; ++i) {
        int rc = derive(&p[i], &c->img[i], nullptr, nullptr);
        if (rc) {
            delete c;
            return rc;
        }
        c->max_nbins = std::max(c->max_nbins, c->img[i].nbins);
    }
    c->io.assign(n, IoEntry{nullptr, 0, nullptr});
    c->cur.assign(n, 0);
    c->pending.assign(n, -1);
    int rc = from_cuda(cudaGetDevice(&c->device));
    if (!rc) rc = from_cuda(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    for (auto &h : c->img) c->pool_bytes += h.bytes;
    if (!rc) rc = from_cuda(cudaMalloc((void **)&c->pool, c->pool_bytes));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&c->d_imgs, sizeof(DevImage) * n));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&c->d_bar, sizeof(GridBarrier)));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&c->d_err, sizeof(int32_t)));
    if (!rc) rc = from_cuda(cudaMemset(c->d_err, 0, sizeof(int32_t)));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&c->d_steps, sizeof(int32_t)));
    if (!rc) rc = from_cuda(cudaMemset(c->d_steps, 0, sizeof(int32_t)));
    if (!rc) rc = from_cuda(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
    if (!rc) rc = from_cuda(cudaEventCreate(&c->ev0));
    if (!rc) rc = from_cuda(cudaEventCreate(&c->ev1));
    for (int i = 0; i < n && !rc; ++i)
        if (c->img[i].p.color_space == 1) {
            rc = from_cuda(upload_lab_tables(0));
            if (!rc) rc = from_cuda(cudaStreamSynchronize(0));
            break;
        }
    if (!rc) {
        // block edge tables are constant for the context's life
        unsigned char *base = c->pool;
        for (auto &h : c->img) {
            for (int l = 1; l <= h.L && !rc; ++l) {
                rc = from_cuda(cudaMemcpy(base + h.off_xe[l], h.xe[l].data(), h.xe[l].size() * 4,
                                          cudaMemcpyHostToDevice));
                if (!rc)
                    rc = from_cuda(cudaMemcpy(base + h.off_ye[l], h.ye[l].data(), h.ye[l].size() * 4,
                                              cudaMemcpyHostToDevice));
            }
            base += h.bytes;
        }
    }
    if (!rc) {
        fill_dev_images(c);
        rc = from_cuda(cudaMemcpy(c->d_imgs, c->h_imgs.data(), sizeof(DevImage) * n, cudaMemcpyHostToDevice));
    }
    // the largest CTA whose warps' shared scratch fits (a whole SM's warps in
    // one CTA balance a step's units best)
    if (!rc) {
        for (int t : {1024, 512, 256, 128}) {
            c->tune.threads_per_block = t;
            rc = configure_launch(c);
            if (!rc) break;
            cudaGetLastError();  // a size that does not fit is not an error of the call
        }
    }
    if (rc) {
        destroy_ctx(c);
        return rc;
    }
    *out = c;
    return SEEDS_OK;
}

int check_io(const seeds_ctx *c, const uint8_t *const *rgb, const int64_t *strides)
{
    if (!rgb || !strides) return SEEDS_ERR_INVALID;
    for (size_t i = 0; i < c->img.size(); ++i)
        if (!rgb[i] || strides[i] < 3 * (int64_t)c->img[i].p.width) return SEEDS_ERR_INVALID;
    return SEEDS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

// A tuning with its zero fields at their defaults (threads_per_block stays 0:
// the largest CTA that fits); SEEDS_ERR_INVALID for a value out of range.
int normalize_tuning(const seeds_tuning &t, seeds_tuning *out)
{
    seeds_tuning n = t;
    if (n.small_block_area == 0) n.small_block_area = 16;
    if (n.pixel_tile_rows == 0) n.pixel_tile_rows = 4;
    if (n.pixel_tile_rows != 2 && n.pixel_tile_rows != 4) return SEEDS_ERR_INVALID;
    if (n.threads_per_block != 0 && n.threads_per_block != 128 && n.threads_per_block != 256 &&
        n.threads_per_block != 512 && n.threads_per_block != 1024)
        return SEEDS_ERR_INVALID;
    if (n.blocks_per_sm < 0 || n.hist_layout < 0 || n.hist_layout > 1) return SEEDS_ERR_INVALID;
    if (n.small_block_area < 1 || n.small_block_area > kSmallMax) return SEEDS_ERR_INVALID;
    if (n.block_tiles < 0 || n.block_tiles > 2) return SEEDS_ERR_INVALID;
    *out = n;
    return SEEDS_OK;
}

extern "C" {

int seeds_plan(const seeds_params *p, int32_t n, const seeds_tuning *t, int32_t sm_count, const int32_t *op_begin,
               const int32_t *op_end, seeds_plan_entry *out, int32_t cap, int32_t *n_entries, int32_t *step_first,
               int64_t *step_threads, int32_t step_cap, int32_t *n_steps)
{
    if (!p || n <= 0 || n > SEEDS_MAX_BATCH || sm_count <= 0 || !n_entries || !n_steps || cap < 0 || step_cap < 0)
        return SEEDS_ERR_INVALID;
    seeds_tuning tune;
    if (normalize_tuning(t ? *t : seeds_tuning{0, 0, 0, 0, 0, 0}, &tune)) return SEEDS_ERR_INVALID;
    std::vector<DevImage> imgs(n);
    std::vector<int> b(n, 0), e(n);
    std::vector<char> pend(n, 0);
    for (int i = 0; i < n; ++i) {
        ImageHost h;
        const int rc = derive(&p[i], &h, nullptr, nullptr);
        if (rc) return rc;
        imgs[i] = plan_image(h, tune);
        const int nops = (int)h.ops.size();
        b[i] = op_begin ? op_begin[i] : 0;
        e[i] = op_end ? op_end[i] : nops;
        if (b[i] < 0 || e[i] < b[i] || e[i] > nops) return SEEDS_ERR_INVALID;
        // a launch that starts after a phase has that phase's moves pending
        pend[i] = b[i] > 0 && is_phase(h.ops[b[i] - 1].kind);
    }
    std::vector<StepEntry> ent;
    std::vector<int32_t> first;
    std::vector<int64_t> vt;
    build_steps(imgs, b, e, pend, (int64_t)sm_count * 32, tune.block_tiles, ent, first, vt);
    *n_entries = (int32_t)ent.size();
    *n_steps = (int32_t)vt.size();
    if (!out && !step_first && !step_threads) return SEEDS_OK;  // the sizes alone
    if (!out || !step_first || cap < *n_entries || step_cap < *n_steps + 1) return SEEDS_ERR_INVALID;
    for (size_t q = 0; q < ent.size(); ++q) {
        const StepEntry &E = ent[q];
        out[q] = seeds_plan_entry{E.img, E.op, E.level, E.phase, E.opidx, E.units, E.group, E.cphase, E.vt_begin};
    }
    for (size_t s = 0; s < first.size(); ++s) step_first[s] = first[s];
    if (step_threads)
        for (size_t s = 0; s < vt.size(); ++s) step_threads[s] = vt[s];
    return SEEDS_OK;
}

int seeds_params_default(seeds_params *p, int32_t width, int32_t height, int32_t num_superpixels)
{
    if (!p) return SEEDS_ERR_INVALID;
    p->width = width;
    p->height = height;
    p->num_superpixels = num_superpixels;
    p->block_levels = 0;
    p->bins_per_channel = 5;
    p->iters_per_level = 2;
    p->patch = 3;
    p->gamma_num = 1;
    p->gamma_den = 1;
    p->color_space = 0;
    p->means_iters = 0;
    p->compactness = 0;
    p->edge_threshold = 0;
    p->compact_prior = 0;
    int32_t lmax = 0;
    int rc = seeds_feasible_levels(p, &lmax);
    if (rc) return rc;
    p->block_levels = std::min(4, lmax);
    return SEEDS_OK;
}

int seeds_feasible_levels(const seeds_params *p, int32_t *max_levels)
{
    if (!p || !max_levels) return SEEDS_ERR_INVALID;
    seeds_params q = *p;
    q.block_levels = 0;
    int32_t gx = 0, gy = 0;
    int rc = derive(&q, nullptr, &gx, &gy);
    if (rc) return rc;
    int L = 0;
    while (L < kMaxLevels && ((int64_t)gx << (L + 1)) <= p->width && ((int64_t)gy << (L + 1)) <= p->height) ++L;
    *max_levels = L;
    return SEEDS_OK;
}

int seeds_check_params(const seeds_params *p, int32_t *gx, int32_t *gy)
{
    int32_t a = 0, b = 0;
    int rc = derive(p, nullptr, &a, &b);
    if (gx) *gx = a;
    if (gy) *gy = b;
    return rc;
}

int seeds_footprint(const seeds_params *p, int32_t n, int64_t *bytes)
{
    if (!p || !bytes || n < 1) return SEEDS_ERR_INVALID;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        ImageHost h;
        int rc = derive(&p[i], &h, nullptr, nullptr);
        if (rc) return rc;
        total += (int64_t)h.bytes + sizeof(DevImage) + 8;
    }
    *bytes = total;
    return SEEDS_OK;
}

int seeds_create(const seeds_params *p, seeds_ctx **out) { return create_ctx(p, 1, out); }

int seeds_batch_create(const seeds_params *p, int32_t n, seeds_ctx **out) { return create_ctx(p, n, out); }

int seeds_destroy(seeds_ctx *c)
{
    if (!c) return SEEDS_ERR_INVALID;
    destroy_ctx(c);
    return SEEDS_OK;
}

int seeds_num_superpixels(const seeds_ctx *c, int32_t *k_out) { return seeds_batch_num_superpixels(c, 0, k_out); }

int seeds_batch_size(const seeds_ctx *c, int32_t *n_out)
{
    if (!c || !n_out) return SEEDS_ERR_INVALID;
    *n_out = (int32_t)c->img.size();
    return SEEDS_OK;
}

int seeds_batch_num_superpixels(const seeds_ctx *c, int32_t i, int32_t *k_out)
{
    if (!c || !k_out || i < 0 || i >= (int32_t)c->img.size()) return SEEDS_ERR_INVALID;
    *k_out = c->img[i].K;
    return SEEDS_OK;
}

int seeds_iterate(seeds_ctx *c, const uint8_t *d_rgb, int64_t row_stride_bytes, void *stream)
{
    if (!c || c->img.size() != 1) return SEEDS_ERR_INVALID;
    return seeds_batch_iterate(c, &d_rgb, &row_stride_bytes, stream);
}

int seeds_labels(seeds_ctx *c, int32_t *d_labels_out, void *stream)
{
    if (!c || c->img.size() != 1) return SEEDS_ERR_INVALID;
    return seeds_batch_labels(c, &d_labels_out, stream);
}

int seeds_batch_iterate(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides, void *stream)
{
    if (!c) return SEEDS_ERR_INVALID;
    int rc = check_io(c, h_rgb_ptrs, h_row_strides);
    if (rc) return rc;
    for (size_t i = 0; i < c->img.size(); ++i) {
        c->io[i].rgb = h_rgb_ptrs[i];
        c->io[i].stride = h_row_strides[i];
    }
    return launch(c, SCHED_ITERATE, 0, 0, (cudaStream_t)stream);
}

int seeds_batch_labels(seeds_ctx *c, int32_t *const *h_label_ptrs, void *stream)
{
    if (!c || !h_label_ptrs || c->stopped_state) return SEEDS_ERR_INVALID;
    for (size_t i = 0; i < c->img.size(); ++i) {
        if (!h_label_ptrs[i]) return SEEDS_ERR_INVALID;
        c->io[i].out = h_label_ptrs[i];
    }
    return launch(c, SCHED_OUTPUT, 0, 0, (cudaStream_t)stream);
}

int seeds_batch_run(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                    int32_t *const *h_label_ptrs, void *stream)
{
    if (!c || !h_label_ptrs) return SEEDS_ERR_INVALID;
    int rc = check_io(c, h_rgb_ptrs, h_row_strides);
    if (rc) return rc;
    for (size_t i = 0; i < c->img.size(); ++i) {
        if (!h_label_ptrs[i]) return SEEDS_ERR_INVALID;
        c->io[i].rgb = h_rgb_ptrs[i];
        c->io[i].stride = h_row_strides[i];
        c->io[i].out = h_label_ptrs[i];
    }
    return launch(c, SCHED_FULL, 0, 0, (cudaStream_t)stream);
}

int seeds_batch_run_anytime(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                            int32_t *const *h_label_ptrs, int32_t max_steps, int64_t budget_ns, void *stream)
{
    if (!c || !h_label_ptrs || max_steps < 0 || budget_ns < 0) return SEEDS_ERR_INVALID;
    int rc = check_io(c, h_rgb_ptrs, h_row_strides);
    if (rc) return rc;
    for (size_t i = 0; i < c->img.size(); ++i) {
        if (!h_label_ptrs[i]) return SEEDS_ERR_INVALID;
        c->io[i].rgb = h_rgb_ptrs[i];
        c->io[i].stride = h_row_strides[i];
        c->io[i].out = h_label_ptrs[i];
    }
    // no limit at all runs every step (and still counts them)
    if (max_steps == 0 && budget_ns == 0) max_steps = INT32_MAX;
    return launch(c, SCHED_FULL, 0, 0, (cudaStream_t)stream, max_steps, budget_ns);
}

int seeds_anytime_steps(seeds_ctx *c, int32_t *steps)
{
    if (!c || !steps) return SEEDS_ERR_INVALID;
    if (c->launched) {
        int rc = from_cuda(cudaEventSynchronize(c->done));
        if (rc) return rc;
    }
    return from_cuda(cudaMemcpy(steps, c->d_steps, sizeof(int32_t), cudaMemcpyDeviceToHost));
}

}  // extern "C"

namespace {

bool host_io_valid(const seeds_ctx *c, const uint8_t *const *h_rgb, const int64_t *h_row_strides,
                   int32_t *const *h_labels, size_t count)
{
    const size_t n = c->img.size();
    for (size_t j = 0; j < count; ++j)
        if (!h_rgb[j] || !h_labels[j] || h_row_strides[j] < 3 * (int64_t)c->img[j % n].p.width) return false;
    return true;
}

// Staging slot `slot` (each slot: every image's RGB, then its int32 labels)
int ensure_stage(seeds_ctx *c, int slot)
{
    const size_t n = c->img.size();
    if (c->stage_rgb.empty()) {
        size_t off = 0;
        c->stage_rgb.resize(n);
        c->stage_out.resize(n);
        for (size_t i = 0; i < n; ++i) {
            c->stage_rgb[i] = off;
            off = align_up(off + (size_t)c->img[i].N * 3);
            c->stage_out[i] = off;
            off = align_up(off + (size_t)c->img[i].N * 4);
        }
        c->stage_bytes = off;
    }
    if (c->stage[slot]) return SEEDS_OK;
    return from_cuda(cudaMalloc((void **)&c->stage[slot], c->stage_bytes));
}

// batch `h_*[0..n)` host -> staging slot, on stream s; points the io records at the slot
int stage_in(seeds_ctx *c, int slot, const uint8_t *const *h_rgb, const int64_t *h_row_strides, cudaStream_t s)
{
    for (size_t i = 0; i < c->img.size(); ++i) {
        const ImageHost &h = c->img[i];
        const size_t row = (size_t)h.p.width * 3;
        int rc = from_cuda(cudaMemcpy2DAsync(c->stage[slot] + c->stage_rgb[i], row, h_rgb[i], (size_t)h_row_strides[i],
                                             row, (size_t)h.p.height, cudaMemcpyHostToDevice, s));
        if (rc) return rc;
        c->io[i].rgb = c->stage[slot] + c->stage_rgb[i];
        c->io[i].stride = (int64_t)row;
        c->io[i].out = (int32_t *)(c->stage[slot] + c->stage_out[i]);
    }
    return SEEDS_OK;
}

int stage_out(seeds_ctx *c, int slot, int32_t *const *h_labels, cudaStream_t s)
{
    for (size_t i = 0; i < c->img.size(); ++i) {
        int rc = from_cuda(cudaMemcpyAsync(h_labels[i], c->stage[slot] + c->stage_out[i], (size_t)c->img[i].N * 4,
                                           cudaMemcpyDeviceToHost, s));
        if (rc) return rc;
    }
    return SEEDS_OK;
}

int ensure_pipe(seeds_ctx *c)
{
    if (c->s_in) return SEEDS_OK;
    int rc = from_cuda(cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking));
    if (!rc) rc = from_cuda(cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&c->ev_entry, &c->ev_in[0], &c->ev_in[1], &c->ev_k[0], &c->ev_k[1], &c->ev_out[0],
                           &c->ev_out[1]})
        if (!rc) rc = from_cuda(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return rc;
}

}  // namespace

extern "C" {

int seeds_run_host(seeds_ctx *c, const uint8_t *const *h_rgb, const int64_t *h_row_strides, int32_t *const *h_labels,
                   void *stream)
{
    if (!c || !h_rgb || !h_row_strides || !h_labels) return SEEDS_ERR_INVALID;
    if (!host_io_valid(c, h_rgb, h_row_strides, h_labels, c->img.size())) return SEEDS_ERR_INVALID;
    int rc = ensure_stage(c, 0);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = stage_in(c, 0, h_rgb, h_row_strides, s);
    if (!rc) rc = launch(c, SCHED_FULL, 0, 0, s);
    if (!rc) rc = stage_out(c, 0, h_labels, s);
    return rc ? rc : from_cuda(cudaEventRecord(c->done, s));
}

// Batch b uses staging slot b & 1.  Its copies in (stream s_in) wait for the
// launch of batch b-2, the last reader of that slot's RGB; its launch (the
// caller's stream) waits for them and for the copies out of batch b-2, the
// last readers of the slot's labels; its copies out (s_out) wait for the
// launch.  Each wait names the event's latest record, made one or two
// batches earlier, before the event is recorded again.
int seeds_run_host_stream(seeds_ctx *c, int32_t n_batches, const uint8_t *const *h_rgb,
                          const int64_t *h_row_strides, int32_t *const *h_labels, void *stream)
{
    if (!c || n_batches < 1 || !h_rgb || !h_row_strides || !h_labels) return SEEDS_ERR_INVALID;
    const size_t n = c->img.size();
    if (!host_io_valid(c, h_rgb, h_row_strides, h_labels, n * (size_t)n_batches)) return SEEDS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    int rc = from_cuda(cudaStreamIsCapturing(s, &cap));
    if (rc) return rc;
    if (cap != cudaStreamCaptureStatusNone) return SEEDS_ERR_INVALID;
    rc = ensure_stage(c, 0);
    if (!rc) rc = ensure_stage(c, 1);
    if (!rc) rc = ensure_pipe(c);
    if (rc) return rc;
    // the copy streams start after the caller's earlier work (an earlier
    // host run may still be reading slot 0)
    rc = from_cuda(cudaEventRecord(c->ev_entry, s));
    if (!rc) rc = from_cuda(cudaStreamWaitEvent(c->s_in, c->ev_entry, 0));
    if (!rc) rc = from_cuda(cudaStreamWaitEvent(c->s_out, c->ev_entry, 0));
    for (int32_t b = 0; b < n_batches && !rc; ++b) {
        const int slot = b & 1;
        const size_t at = (size_t)b * n;
        if (b >= 2) rc = from_cuda(cudaStreamWaitEvent(c->s_in, c->ev_k[slot], 0));
        if (!rc) rc = stage_in(c, slot, h_rgb + at, h_row_strides + at, c->s_in);
        if (!rc) rc = from_cuda(cudaEventRecord(c->ev_in[slot], c->s_in));
        if (!rc) rc = from_cuda(cudaStreamWaitEvent(s, c->ev_in[slot], 0));
        if (!rc && b >= 2) rc = from_cuda(cudaStreamWaitEvent(s, c->ev_out[slot], 0));
        if (!rc) rc = launch(c, SCHED_FULL, 0, 0, s);
        if (!rc) rc = from_cuda(cudaEventRecord(c->ev_k[slot], s));
        if (!rc) rc = from_cuda(cudaStreamWaitEvent(c->s_out, c->ev_k[slot], 0));
        if (!rc) rc = stage_out(c, slot, h_labels + at, c->s_out);
        if (!rc) rc = from_cuda(cudaEventRecord(c->ev_out[slot], c->s_out));
    }
    // the caller's stream ends after the last copies out (s_out runs them in order)
    const int last = (n_batches - 1) & 1;
    if (!rc) rc = from_cuda(cudaStreamWaitEvent(s, c->ev_out[last], 0));
    return rc ? rc : from_cuda(cudaEventRecord(c->done, s));
}

int seeds_status(seeds_ctx *c)
{
    if (!c) return SEEDS_ERR_INVALID;
    if (c->launched) {
        int rc = from_cuda(cudaEventSynchronize(c->done));
        if (rc) return rc;
    }
    int32_t e = 0;
    int rc = from_cuda(cudaMemcpy(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (rc) return rc;
    if (e != 0) {
        cudaMemset(c->d_err, 0, sizeof(int32_t));
        return SEEDS_ERR_DEVICE;
    }
    return from_cuda(cudaGetLastError());
}

int seeds_set_tuning(seeds_ctx *c, const seeds_tuning *t)
{
    if (!c || !t) return SEEDS_ERR_INVALID;
    seeds_tuning n;
    if (normalize_tuning(*t, &n)) return SEEDS_ERR_INVALID;
    if (c->launched) cudaEventSynchronize(c->done);
    const seeds_tuning old = c->tune;
    auto apply = [&](const seeds_tuning &v) {
        c->tune = v;
        free_schedules(c);
        fill_dev_images(c);
        int rc = from_cuda(cudaMemcpy(c->d_imgs, c->h_imgs.data(), sizeof(DevImage) * c->img.size(),
                                      cudaMemcpyHostToDevice));
        return rc ? rc : configure_launch(c);
    };
    int rc = SEEDS_ERR_INVALID;
    if (n.threads_per_block != 0) {
        rc = apply(n);
    } else {  // the default: the largest CTA that fits
        for (int threads : {1024, 512, 256, 128}) {
            n.threads_per_block = threads;
            rc = apply(n);
            if (!rc) break;
            cudaGetLastError();
        }
    }
    if (rc) {  // a setting that cannot launch leaves the context as it was
        apply(old);
        cudaGetLastError();
    }
    return rc;
}

int seeds_autotune(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides,
                   int32_t *const *h_label_ptrs, int32_t reps, void *stream, seeds_tuning *best)
{
    if (!c || reps < 1) return SEEDS_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = from_cuda(cudaEventCreate(&a));
    if (!rc) rc = from_cuda(cudaEventCreate(&b));
    // best-of-reps time of one batch under a setting; +inf if it cannot run
    auto time_it = [&](const seeds_tuning &t, float *ms) -> int {
        *ms = 1e30f;
        if (seeds_set_tuning(c, &t) != SEEDS_OK) return SEEDS_OK;
        int r = seeds_batch_run(c, h_rgb_ptrs, h_row_strides, h_label_ptrs, stream);
        for (int i = 0; i < reps && !r; ++i) {
            r = from_cuda(cudaEventRecord(a, st));
            if (!r) r = seeds_batch_run(c, h_rgb_ptrs, h_row_strides, h_label_ptrs, stream);
            if (!r) r = from_cuda(cudaEventRecord(b, st));
            if (!r) r = from_cuda(cudaEventSynchronize(b));
            float e = 0.f;
            if (!r) r = from_cuda(cudaEventElapsedTime(&e, a, b));
            if (!r) *ms = std::min(*ms, e);
        }
        return r;
    };
    seeds_tuning cur = c->tune;
    if (!rc) rc = tune_search(c->tune, time_it, &cur);  // coordinate descent, one pass; a change must win by 2%
    if (!rc) rc = seeds_set_tuning(c, &cur);
    if (!rc && best) *best = cur;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return rc;
}

int seeds_tune_search(const seeds_tuning *start, seeds_tune_cost_fn cost, void *user, seeds_tuning *best)
{
    if (!start || !cost || !best) return SEEDS_ERR_INVALID;
    return tune_search(
        *start,
        [&](const seeds_tuning &t, float *ms) {
            *ms = cost(&t, user);
            return SEEDS_OK;
        },
        best);
}

int seeds_get_tuning(const seeds_ctx *c, seeds_tuning *t)
{
    if (!c || !t) return SEEDS_ERR_INVALID;
    *t = c->tune;
    return SEEDS_OK;
}

int seeds_debug_num_ops(const seeds_ctx *c, int32_t i, int32_t *n_ops)
{
    if (!c || !n_ops || i < 0 || i >= (int32_t)c->img.size()) return SEEDS_ERR_INVALID;
    *n_ops = (int32_t)c->img[i].ops.size();
    return SEEDS_OK;
}

int seeds_debug_op_info(const seeds_ctx *c, int32_t i, int32_t op, int32_t *kind, int32_t *level, int32_t *phase)
{
    if (!c || i < 0 || i >= (int32_t)c->img.size()) return SEEDS_ERR_INVALID;
    const auto &ops = c->img[i].ops;
    if (op < 0 || op >= (int32_t)ops.size()) return SEEDS_ERR_INVALID;
    if (kind) *kind = ops[op].kind;
    if (level) *level = ops[op].level;
    if (phase) *phase = ops[op].phase;
    return SEEDS_OK;
}

int seeds_debug_run_ops(seeds_ctx *c, const uint8_t *const *h_rgb_ptrs, const int64_t *h_row_strides, int32_t op_begin,
                        int32_t op_end, void *stream)
{
    if (!c || op_begin < 0 || op_end < op_begin) return SEEDS_ERR_INVALID;
    int rc = check_io(c, h_rgb_ptrs, h_row_strides);
    if (rc) return rc;
    for (size_t i = 0; i < c->img.size(); ++i) {
        c->io[i].rgb = h_rgb_ptrs[i];
        c->io[i].stride = h_row_strides[i];
    }
    return launch(c, SCHED_DEBUG, op_begin, op_end, (cudaStream_t)stream);
}

int seeds_debug_read_state(seeds_ctx *c, int32_t i, int32_t level, int32_t *h_labels, int32_t *h_hist,
                           int32_t *h_sizes, int32_t *h_bins)
{
    if (!c || i < 0 || i >= (int32_t)c->img.size()) return SEEDS_ERR_INVALID;
    const ImageHost &h = c->img[i];
    const DevImage &d = c->h_imgs[i];
    if (level < 0 || level > h.L) return SEEDS_ERR_INVALID;
    int rc = from_cuda(cudaDeviceSynchronize());
    if (rc) return rc;
    const int q = c->cur[i] & 1;  // buffer holding the complete state
    if (h_labels) {
        const size_t n = (size_t)h.nbx[level] * h.nby[level];
        std::vector<uint16_t> t(n);
        rc = from_cuda(cudaMemcpy(t.data(), d.lab[level][q], n * 2, cudaMemcpyDeviceToHost));
        if (rc) return rc;
        for (size_t q = 0; q < n; ++q) h_labels[q] = t[q];
    }
    if (h_hist) {
        const size_t n = (size_t)h.K * h.nbins;
        std::vector<int32_t> t(n);
        rc = from_cuda(cudaMemcpy(t.data(), d.hist[q], n * 4, cudaMemcpyDeviceToHost));
        if (rc) return rc;
        for (int k = 0; k < h.K; ++k)
            for (int j = 0; j < h.nbins; ++j)
                h_hist[(size_t)k * h.nbins + j] = d.hist_jmajor ? t[(size_t)j * h.K + k] : t[(size_t)k * h.nbins + j];
    }
    if (h_sizes) {
        rc = from_cuda(cudaMemcpy(h_sizes, d.size[q], (size_t)h.K * 4, cudaMemcpyDeviceToHost));
        if (rc) return rc;
    }
    if (h_bins) {
        if (d.bins16) {
            std::vector<uint16_t> t((size_t)h.N);
            rc = from_cuda(cudaMemcpy(t.data(), d.bins, (size_t)h.N * 2, cudaMemcpyDeviceToHost));
            if (rc) return rc;
            for (int64_t q = 0; q < h.N; ++q) h_bins[q] = t[q];
        } else {
            std::vector<uint8_t> t((size_t)h.N);
            rc = from_cuda(cudaMemcpy(t.data(), d.bins, (size_t)h.N, cudaMemcpyDeviceToHost));
            if (rc) return rc;
            for (int64_t q = 0; q < h.N; ++q) h_bins[q] = t[q];
        }
    }
    return SEEDS_OK;
}

int seeds_debug_set_labels(seeds_ctx *c, int32_t i, int32_t level, const int32_t *h_labels)
{
    if (!c || !h_labels || i < 0 || i >= (int32_t)c->img.size()) return SEEDS_ERR_INVALID;
    const ImageHost &h = c->img[i];
    if (level < 0 || level > h.L) return SEEDS_ERR_INVALID;
    const size_t n = (size_t)h.nbx[level] * h.nby[level];
    std::vector<uint16_t> t(n);
    for (size_t q = 0; q < n; ++q) {
        if (h_labels[q] < 0 || h_labels[q] >= h.K) return SEEDS_ERR_INVALID;
        t[q] = (uint16_t)h_labels[q];
    }
    int rc = from_cuda(cudaDeviceSynchronize());
    for (int q = 0; q < 2 && !rc; ++q)
        rc = from_cuda(cudaMemcpy(c->h_imgs[i].lab[level][q], t.data(), n * 2, cudaMemcpyHostToDevice));
    if (!rc) rc = from_cuda(launch_recount(c->d_imgs, i, level, h.N, 0));
    if (!rc) rc = from_cuda(cudaDeviceSynchronize());
    c->launches += 2;
    c->pending[i] = -1;  // the injected state replaces any moves awaiting catch-up
    return rc;
}

int seeds_debug_inject_error(seeds_ctx *c)
{
    if (!c) return SEEDS_ERR_INVALID;
    const int32_t v = DERR_INJECTED;
    return from_cuda(cudaMemcpy(c->d_err, &v, sizeof(v), cudaMemcpyHostToDevice));
}

int seeds_debug_barrier_test(seeds_ctx *c, int64_t timeout_ns, int32_t withhold_step)
{
    if (!c || timeout_ns < 0 || withhold_step < -1) return SEEDS_ERR_INVALID;
    c->dbg_timeout_ns = (unsigned long long)timeout_ns;
    c->dbg_withhold = withhold_step + 1;
    return SEEDS_OK;
}

int seeds_debug_launch_count(const seeds_ctx *c, int64_t *n)
{
    if (!c || !n) return SEEDS_ERR_INVALID;
    *n = c->launches;
    return SEEDS_OK;
}

int seeds_profile_enable(seeds_ctx *c, int32_t enable)
{
    if (!c) return SEEDS_ERR_INVALID;
    if (enable && !c->d_trace) {
        int most = 0;
        for (auto &h : c->img) most = std::max(most, (int)h.ops.size());
        c->trace_cap = 1 + most;
        int rc = from_cuda(cudaMalloc((void **)&c->d_trace, sizeof(unsigned long long) * c->trace_cap));
        if (rc) return rc;
    }
    c->profile = enable != 0;
    return SEEDS_OK;
}

int seeds_profile_steps(seeds_ctx *c, int64_t *h_ns, int32_t cap, int32_t *n)
{
    if (!c || !n || !c->profiled || c->traced_steps == 0) return SEEDS_ERR_INVALID;
    const int m = 1 + c->traced_steps;
    *n = m;
    if (!h_ns || cap < m) return SEEDS_OK;
    int rc = from_cuda(cudaEventSynchronize(c->ev1));
    if (rc) return rc;
    std::vector<unsigned long long> t(m);
    rc = from_cuda(cudaMemcpy(t.data(), c->d_trace, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
    if (rc) return rc;
    for (int i = 0; i < m; ++i) h_ns[i] = (int64_t)(t[i] - t[0]);
    return SEEDS_OK;
}

int seeds_profile_last_ms(seeds_ctx *c, float *ms)
{
    if (!c || !ms || !c->profiled) return SEEDS_ERR_INVALID;
    int rc = from_cuda(cudaEventSynchronize(c->ev1));
    if (rc) return rc;
    return from_cuda(cudaEventElapsedTime(ms, c->ev0, c->ev1));
}

}  // extern "C"
