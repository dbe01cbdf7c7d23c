// seeds_server.cu -- continuous-batching serving runtime behind the
// seeds_server_* entry points of include/seeds.h.
//
// A server owns one device arena, a table of image slots and a stream.
// Requests wait in a FIFO queue and are admitted when a slot is free and
// their state fits the arena (first-fit allocator with coalescing).  Every
// call to seeds_server_step launches one epoch: one persistent-kernel launch
// that advances every resident image by up to `epoch_steps` of its ops, so
// images admitted while others are on the device start at the next epoch
// and run side by side with them.  The copies run on two streams beside
// the launches: an admitted image's RGB goes in while the previous epoch
// runs, and a finished image's labels go out while the next one does.  A
// finished image's arena space returns to the allocator only once its
// epoch's copies out have completed, so a later admission's copy in, which
// waits for nothing, never overwrites state still in use.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "seeds.h"
#include "seeds_device.cuh"
#include "seeds_host.h"

using namespace seeds;
using namespace seeds::host;

namespace {

// First-fit allocator over [0, size) with coalescing of neighbouring holes.
class ArenaAllocator {
  public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const
    {
        size_t t = 0;
        for (auto &kv : free_) t += kv.second;
        return t;
    }

  private:
    std::map<size_t, size_t> free_;  // offset -> length
};

struct Request {
    int64_t id = 0;
    ImageHost h;
    const uint8_t *h_rgb = nullptr;
    int64_t stride = 0;
    int32_t *h_out = nullptr;
    size_t off = 0, bytes = 0, rgb_off = 0, out_off = 0;
    int slot = -1, progress = 0, pending = -1, nops = 0;
};

struct Epoch {
    cudaEvent_t ev = nullptr;   // recorded after the epoch's copies out
    std::vector<int64_t> done;  // requests whose labels this epoch delivers
    std::vector<std::pair<size_t, size_t>> freed;  // their arena space (offset, bytes)
};

// bytes a request occupies in the arena: its state, its image, its labels
size_t request_bytes(const ImageHost &h, size_t *rgb_off, size_t *out_off)
{
    size_t off = h.bytes;
    *rgb_off = off;
    off = align_up(off + (size_t)h.N * 3);
    *out_off = off;
    off = align_up(off + (size_t)h.N * 4);
    return off;
}

}  // namespace

struct seeds_server {
    int device = 0, sm_count = 0;
    seeds_server_config cfg{};
    // Block phases stay per unit (block_tiles 1): an epoch's step mixes
    // images at different levels, and the tile rule, which decides per step,
    // would also tile the levels of small images with large blocks, whose
    // warps then judge a tile's boundary blocks one after another for longer
    // than the rest of the step takes.
    seeds_tuning tune{1024, 0, 0, 16, 4, 1};
    int max_nbins = 1;
    unsigned char *arena = nullptr;
    ArenaAllocator alloc;
    DevImage *d_imgs = nullptr;
    GridBarrier *d_bar = nullptr;
    int32_t *d_err = nullptr;
    StepEntry *d_ent = nullptr;
    int32_t *d_first = nullptr;
    int64_t *d_vt = nullptr;
    cudaStream_t stream = nullptr;            // the epochs' launches
    cudaStream_t s_in = nullptr, s_out = nullptr;  // copies in and out
    cudaEvent_t ev_in = nullptr, ev_k = nullptr;   // copies in done; launch done
    int grid = 0;
    size_t smem = 0;
    std::deque<Request *> queue;
    std::vector<Request *> slots;
    std::deque<Epoch> inflight;
    std::vector<cudaEvent_t> spare_events;
    cudaEvent_t t0 = nullptr;
    std::chrono::steady_clock::time_point h0;
    std::vector<std::pair<int64_t, float>> completed;
    int64_t next_id = 0, epochs = 0, launches = 0, admitted = 0;
};

namespace {

cudaEvent_t take_event(seeds_server *s)
{
    if (!s->spare_events.empty()) {
        cudaEvent_t e = s->spare_events.back();
        s->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// move finished epochs' requests to the completed list; block on the oldest
// epoch while more than `keep` are in flight
int reap(seeds_server *s, size_t keep)
{
    while (!s->inflight.empty()) {
        Epoch &ep = s->inflight.front();
        cudaError_t q = cudaEventQuery(ep.ev);
        if (q == cudaErrorNotReady) {
            if (s->inflight.size() <= keep) return SEEDS_OK;
            q = cudaEventSynchronize(ep.ev);
        }
        if (q != cudaSuccess) return from_cuda(q);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->t0, ep.ev);
        for (int64_t id : ep.done) s->completed.emplace_back(id, ms);
        for (auto &f : ep.freed) s->alloc.release(f.first, f.second);
        s->spare_events.push_back(ep.ev);
        s->inflight.pop_front();
    }
    return SEEDS_OK;
}

void destroy_server(seeds_server *s)
{
    if (!s) return;
    for (cudaStream_t st : {s->stream, s->s_in, s->s_out})
        if (st) cudaStreamSynchronize(st);
    for (auto *r : s->queue) delete r;
    for (auto *r : s->slots) delete r;
    for (auto &ep : s->inflight) cudaEventDestroy(ep.ev);
    for (auto e : s->spare_events) cudaEventDestroy(e);
    if (s->t0) cudaEventDestroy(s->t0);
    cudaFree(s->arena);
    cudaFree(s->d_imgs);
    cudaFree(s->d_bar);
    cudaFree(s->d_err);
    cudaFree(s->d_ent);
    cudaFree(s->d_first);
    cudaFree(s->d_vt);
    for (cudaStream_t st : {s->stream, s->s_in, s->s_out})
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : {s->ev_in, s->ev_k})
        if (e) cudaEventDestroy(e);
    delete s;
}

}  // namespace

extern "C" {

int seeds_server_create(const seeds_server_config *cfg, seeds_server **out)
{
    if (!cfg || !out) return SEEDS_ERR_INVALID;
    *out = nullptr;
    if (cfg->arena_bytes < (1 << 20) || cfg->max_slots < 1 || cfg->max_slots > kMaxEpochSlots ||
        cfg->epoch_steps < 1 || cfg->epoch_steps > 1024 || cfg->max_bins_per_channel < 1 ||
        cfg->max_bins_per_channel > 16)
        return SEEDS_ERR_INVALID;
    seeds_server *s = new (std::nothrow) seeds_server;
    if (!s) return SEEDS_ERR_NO_MEMORY;
    s->cfg = *cfg;
    const int B = cfg->max_bins_per_channel;
    s->max_nbins = B * B * B;
    s->slots.assign(cfg->max_slots, nullptr);
    s->alloc.reset((size_t)cfg->arena_bytes);
    const size_t max_ent = (size_t)cfg->epoch_steps * 2 * cfg->max_slots;
    int rc = from_cuda(cudaGetDevice(&s->device));
    if (!rc) rc = from_cuda(cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device));
    if (!rc) rc = from_cuda(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    if (!rc) rc = from_cuda(cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking));
    if (!rc) rc = from_cuda(cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking));
    if (!rc) rc = from_cuda(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
    if (!rc) rc = from_cuda(cudaEventCreateWithFlags(&s->ev_k, cudaEventDisableTiming));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->arena, (size_t)cfg->arena_bytes));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->d_imgs, sizeof(DevImage) * cfg->max_slots));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->d_bar, sizeof(GridBarrier)));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->d_err, sizeof(int32_t)));
    if (!rc) rc = from_cuda(cudaMemset(s->d_err, 0, sizeof(int32_t)));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->d_ent, sizeof(StepEntry) * max_ent));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->d_first, sizeof(int32_t) * (cfg->epoch_steps + 1)));
    if (!rc) rc = from_cuda(cudaMalloc((void **)&s->d_vt, sizeof(int64_t) * cfg->epoch_steps));
    if (!rc) rc = from_cuda(upload_lab_tables(0));
    if (!rc) rc = from_cuda(cudaStreamSynchronize(0));
    if (!rc) {
        // the largest CTA whose warps' shared scratch fits
        for (int threads : {1024, 512, 256, 128}) {
            s->tune.threads_per_block = threads;
            s->smem = (size_t)(threads / 32) * warp_scratch_bytes(s->max_nbins);
            int per_sm = 0;
            rc = from_cuda(prepare_persistent(s->smem));
            if (!rc) rc = from_cuda(persistent_max_blocks_per_sm(threads, s->smem, &per_sm));
            if (!rc && per_sm < 1) rc = SEEDS_ERR_INVALID;
            s->grid = per_sm * s->sm_count;
            if (!rc) break;
            cudaGetLastError();  // a size that does not fit is not an error of the call
        }
    }
    if (!rc) rc = from_cuda(cudaEventCreate(&s->t0));
    if (!rc) rc = from_cuda(cudaEventRecord(s->t0, s->stream));
    if (!rc) rc = from_cuda(cudaEventSynchronize(s->t0));
    if (rc) {
        destroy_server(s);
        return rc;
    }
    s->h0 = std::chrono::steady_clock::now();
    *out = s;
    return SEEDS_OK;
}

int seeds_server_destroy(seeds_server *s)
{
    if (!s) return SEEDS_ERR_INVALID;
    destroy_server(s);
    return SEEDS_OK;
}

int seeds_server_submit(seeds_server *s, const seeds_params *p, const uint8_t *h_rgb, int64_t row_stride_bytes,
                        int32_t *h_labels, int64_t *id_out)
{
    if (!s || !p || !h_rgb || !h_labels || !id_out) return SEEDS_ERR_INVALID;
    if (row_stride_bytes < 3 * (int64_t)p->width) return SEEDS_ERR_INVALID;
    if (p->bins_per_channel > s->cfg.max_bins_per_channel) return SEEDS_ERR_INVALID;
    Request *r = new (std::nothrow) Request;
    if (!r) return SEEDS_ERR_NO_MEMORY;
    int rc = derive(p, &r->h, nullptr, nullptr);
    if (rc) {
        delete r;
        return rc;
    }
    r->bytes = request_bytes(r->h, &r->rgb_off, &r->out_off);
    if (r->bytes > (size_t)s->cfg.arena_bytes) {  // could never be admitted
        delete r;
        return SEEDS_ERR_NO_MEMORY;
    }
    r->h_rgb = h_rgb;
    r->stride = row_stride_bytes;
    r->h_out = h_labels;
    r->nops = (int)r->h.ops.size();
    r->id = s->next_id++;
    s->queue.push_back(r);
    *id_out = r->id;
    return SEEDS_OK;
}

int seeds_server_step(seeds_server *s, int32_t *resident_out)
{
    if (!s) return SEEDS_ERR_INVALID;
    int rc = reap(s, 2);  // at most two epochs queued ahead of the device
    if (rc) return rc;
    cudaStream_t st = s->stream;

    // admit from the head of the queue while a slot and arena space are free
    int admitted_now = 0;
    while (!s->queue.empty()) {
        Request *r = s->queue.front();
        int slot = -1;
        for (int i = 0; i < (int)s->slots.size(); ++i)
            if (!s->slots[i]) {
                slot = i;
                break;
            }
        if (slot < 0 || !s->alloc.alloc(r->bytes, &r->off)) break;
        s->queue.pop_front();
        unsigned char *base = s->arena + r->off;
        const size_t row = (size_t)r->h.p.width * 3;
        rc = from_cuda(cudaMemcpy2DAsync(base + r->rgb_off, row, r->h_rgb, (size_t)r->stride, row,
                                         (size_t)r->h.p.height, cudaMemcpyHostToDevice, s->s_in));
        const DevImage rec =
            make_dev_image(r->h, base, s->tune, IoEntry{base + r->rgb_off, (int64_t)row, (int32_t *)(base + r->out_off)},
                           s->d_err);
        if (!rc) rc = from_cuda(launch_admit(s->d_imgs, slot, rec, st));
        if (rc) {
            cudaStreamSynchronize(s->s_in);  // its copy in may be under way
            s->alloc.release(r->off, r->bytes);
            delete r;
            break;
        }
        ++s->launches;
        r->slot = slot;
        s->slots[slot] = r;
        ++s->admitted;
        ++admitted_now;
    }
    // the epoch reads the admitted images' RGB (also after a failed
    // admission: the ones admitted before it stay resident)
    if (admitted_now) {
        int rw = from_cuda(cudaEventRecord(s->ev_in, s->s_in));
        if (!rw) rw = from_cuda(cudaStreamWaitEvent(st, s->ev_in, 0));
        if (!rc) rc = rw;
    }
    if (rc) return rc;

    // plan the epoch: every resident image advances by up to epoch_steps ops
    EpochPlan plan;
    std::memset(&plan, 0, sizeof(plan));
    plan.split_below = s->sm_count * 32;
    plan.tile_policy = s->tune.block_tiles;
    for (Request *r : s->slots) {
        if (!r) continue;
        EpochSlot &q = plan.s[plan.n++];
        q.slot = r->slot;
        q.begin = r->progress;
        q.end = std::min(r->progress + s->cfg.epoch_steps, r->nops);
        q.catchup = r->progress > 0 && r->pending == r->progress - 1;
        plan.nsteps = std::max(plan.nsteps, q.end - q.begin);
    }
    if (resident_out) *resident_out = plan.n;
    if (plan.n == 0) return SEEDS_OK;
    rc = from_cuda(launch_epoch_schedule(s->d_imgs, plan, s->d_ent, s->d_first, s->d_vt, st));
    if (!rc) rc = from_cuda(cudaMemsetAsync(s->d_bar, 0, sizeof(GridBarrier), st));
    Schedule sch{};
    sch.ent = s->d_ent;
    sch.step_first = s->d_first;
    sch.step_vt = s->d_vt;
    sch.nsteps = plan.nsteps;
    sch.max_nbins = s->max_nbins;
    sch.trace = nullptr;
    if (!rc)
        rc = from_cuda(
            launch_persistent(s->d_imgs, sch, s->d_bar, s->d_err, s->grid, s->tune.threads_per_block, s->smem, st));
    if (!rc) rc = from_cuda(cudaEventRecord(s->ev_k, st));
    if (!rc) rc = from_cuda(cudaStreamWaitEvent(s->s_out, s->ev_k, 0));
    if (rc) return rc;
    s->launches += 2;
    ++s->epochs;

    // deliver the images that finished in this epoch
    Epoch ep;
    for (int i = 0; i < plan.n; ++i) {
        Request *r = s->slots[plan.s[i].slot];
        r->progress = plan.s[i].end;
        r->pending = is_phase(r->h.ops[r->progress - 1].kind) ? r->progress - 1 : -1;
        if (r->progress < r->nops) continue;
        rc = from_cuda(cudaMemcpyAsync(r->h_out, s->arena + r->off + r->out_off, (size_t)r->h.N * 4,
                                       cudaMemcpyDeviceToHost, s->s_out));
        if (rc) return rc;
        ep.done.push_back(r->id);
        ep.freed.emplace_back(r->off, r->bytes);
        s->slots[r->slot] = nullptr;
        delete r;
    }
    ep.ev = take_event(s);
    rc = from_cuda(cudaEventRecord(ep.ev, s->s_out));
    if (rc) return rc;
    s->inflight.push_back(ep);
    return SEEDS_OK;
}

int seeds_server_poll(seeds_server *s, int64_t *ids, float *done_ms, int32_t cap, int32_t *n)
{
    if (!s || !n || cap < 0) return SEEDS_ERR_INVALID;
    int rc = reap(s, (size_t)-1);
    if (rc) return rc;
    const int m = std::min<int>(cap, (int)s->completed.size());
    for (int i = 0; i < m; ++i) {
        if (ids) ids[i] = s->completed[i].first;
        if (done_ms) done_ms[i] = s->completed[i].second;
    }
    s->completed.erase(s->completed.begin(), s->completed.begin() + m);
    *n = m;
    return SEEDS_OK;
}

int seeds_server_drain(seeds_server *s)
{
    if (!s) return SEEDS_ERR_INVALID;
    int rc = SEEDS_OK;
    for (cudaStream_t st : {s->stream, s->s_in, s->s_out})
        if (!rc) rc = from_cuda(cudaStreamSynchronize(st));
    if (rc) return rc;
    rc = reap(s, 0);
    if (rc) return rc;
    int32_t e = 0;
    rc = from_cuda(cudaMemcpy(&e, s->d_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (rc) return rc;
    if (e) {
        cudaMemset(s->d_err, 0, sizeof(int32_t));
        return SEEDS_ERR_DEVICE;
    }
    return SEEDS_OK;
}

int seeds_server_stats(const seeds_server *s, seeds_server_stats_t *out)
{
    if (!s || !out) return SEEDS_ERR_INVALID;
    out->queued = (int32_t)s->queue.size();
    int res = 0;
    for (auto *r : s->slots) res += r != nullptr;
    out->resident = res;
    out->arena_free_bytes = (int64_t)s->alloc.free_bytes();
    out->epochs = s->epochs;
    out->launches = s->launches;
    out->admitted = s->admitted;
    out->host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s->h0).count();
    return SEEDS_OK;
}

}  // extern "C"
