// Serving loop: HiVision's MTVS / IMMF / HPVE pipeline (Sec. 4: tile
// requests are parsed into a first-in-first-out task pool, processed by idle
// workers, completed into a result pool) as one GPU-resident loop.
//
// A native worker thread owns `slots`; each slot is a CUDA stream with a
// pinned request block, device and pinned output buffers of fixed capacity,
// and a completion event.  Requests wait in a FIFO queue.  Whenever a slot is
// free the worker forms a batch from the oldest request's (layer, mode) group,
// admitting requests while the slot's output memory and tile count allow
// (admission by memory), and launches it: request block H2D + render kernel
// (captured CUDA graphs per slot and group: one for small batches, one for
// full ones), then the D2H of the tiles.
// Requests that arrive while other batches run are batched into the next free
// slot, so their work overlaps on the device (continuous batching).  Results
// are handed out zero-copy from the slot's pinned buffer; a slot is recycled
// after the poll that follows the one that exported its last result.
// At submission (Parse Tasks), a request whose tile the layer cannot reach is
// completed at once with an all-zero tile, and, with a result pool, one whose
// tile is in the pool is completed from it; the worker stores every rendered
// tile in the pool.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include <string.h>

#include "hv_device.cuh"
#include "hv_internal.h"

namespace hv {

namespace {

// Batches of at most this many tiles take the small-batch graph.
constexpr uint32_t kSmallBatch = 8;

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Item {
    hv_tile_req req;
    uint64_t tag;
    double t_submit;
    uint64_t seq;          // arrival order
    uint64_t offset = 0;   // output offset in the slot
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t* h_block = nullptr;   // pinned: [uint32 count, pad to 16][requests]
    uint8_t* d_block = nullptr;
    uint8_t* d_out = nullptr;
    uint8_t* h_out = nullptr;     // pinned
    std::vector<Item> items;
    int state = 0;                // 0 free, 1 in flight, 2 results pending poll, 3 exported
    int outstanding = 0;          // results not yet exported
    double t_start = 0;
    int status = HV_OK;
    std::map<uint64_t, cudaGraphExec_t> graphs;   // key: size class << 40 | layer << 8 | mode << 4 | index
};

struct Done {
    uint64_t tag;
    int32_t status;
    uint32_t bytes;
    const uint8_t* data;
    double t_submit, t_start, t_done;
    int slot;                                      // -1: completed at submission
    std::shared_ptr<std::vector<uint8_t>> own;     // a tile from the result pool
};

}  // namespace

struct Server {
    Ctx* ctx;
    std::vector<Layer*> layers;
    hv_server_opts opts;
    uint32_t max_batch;
    uint64_t slot_bytes;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    // the task pool: one FIFO per (layer, mode) group; a batch takes the group
    // holding the oldest request
    std::map<uint32_t, std::deque<Item>> queues;
    uint64_t queued = 0, seq = 0;
    std::deque<Done> done;
    std::vector<int> exported;     // slots whose results the last poll handed out
    std::vector<std::shared_ptr<std::vector<uint8_t>>> held;   // pool tiles the last poll handed out
    std::vector<uint8_t> zeros;    // the all-zero tile of unreachable requests
    ResultPool* pool = nullptr;
    uint64_t pool_hits = 0, empty_tiles = 0;
    std::thread worker;
    bool stopping = false;
    bool failed = false;
    std::string error;
    uint64_t launched = 0, batches = 0, graph_launches = 0;
};

namespace {

int slot_key_index(const Server* S, const hv_tile_req& r) {
    Layer* L = S->layers[r.layer];
    int idx = (S->opts.index_kind == HV_INDEX_LEARNED && (L->indexes & HV_INDEX_LEARNED)) ? HV_INDEX_LEARNED
                                                                                           : HV_INDEX_RTREE;
    return idx;
}

// Launch one batch on slot `k` (worker thread, lock not held).
int launch_batch(Server* S, int k) {
    Slot& sl = S->slots[k];
    const hv_tile_req& r0 = sl.items[0].req;
    Layer* L = S->layers[r0.layer];
    int mode = r0.mode;
    int index = slot_key_index(S, r0);
    uint32_t n = (uint32_t)sl.items.size();
    uint64_t tb = hv_tile_bytes(mode);
    *(uint32_t*)sl.h_block = n;
    hv_tile_req* reqs = (hv_tile_req*)(sl.h_block + 16);
    for (uint32_t i = 0; i < n; i++) {
        reqs[i] = sl.items[i].req;
        sl.items[i].offset = (uint64_t)i * tb;
    }
    const uint64_t block_bytes = 16 + (uint64_t)S->max_batch * sizeof(hv_tile_req);
    const hv_style* style = &S->opts.style;
    if (S->opts.use_graphs) {
        // three graphs per group: a single request and small batches launch a
        // grid sized for one or a few tiles, so that each tile is split into
        // the short strips and column parts (more CTAs per tile) that
        // hv_render_tiles gives such a batch; larger batches launch the grid
        // of a full batch.  The column parts of a single request pay off
        // only on an idle device: with other batches in flight it takes the
        // small-batch grid (measured: at 50,000 requests/s the parts raised
        // p99 from 2.2 to 4.2 ms)
        bool alone = true;
        for (size_t j = 0; j < S->slots.size() && alone; j++)
            if ((int)j != k && __atomic_load_n(&S->slots[j].state, __ATOMIC_RELAXED) == 1) alone = false;
        const uint32_t small = S->max_batch < kSmallBatch ? S->max_batch : kSmallBatch;
        const uint32_t cls = (n == 1 && alone) ? 0u : (n <= small ? 1u : 2u);
        const uint32_t n_cap = cls == 0 ? 1u : (cls == 1 ? small : S->max_batch);
        uint64_t key = ((uint64_t)cls << 40) | ((uint64_t)r0.layer << 8) | ((uint64_t)mode << 4) | (uint64_t)index;
        auto it = sl.graphs.find(key);
        if (it == sl.graphs.end()) {
            cudaGraph_t g;
            HV_CUDA(cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal));
            cudaMemcpyAsync(sl.d_block, sl.h_block, block_bytes, cudaMemcpyHostToDevice, sl.st);
            int rc = launch_render(L, (const hv_tile_req*)(sl.d_block + 16), n_cap, mode, index, style,
                                   sl.d_out, sl.st, nullptr, (const uint32_t*)sl.d_block);
            cudaError_t e = cudaStreamEndCapture(sl.st, &g);
            if (rc != HV_OK) return rc;
            HV_CUDA(e);
            cudaGraphExec_t ge;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            HV_CUDA(e);
            it = sl.graphs.emplace(key, ge).first;
        }
        HV_CUDA(cudaGraphLaunch(it->second, sl.st));
        S->graph_launches++;
    } else {
        HV_CUDA(cudaMemcpyAsync(sl.d_block, sl.h_block, 16 + (uint64_t)n * sizeof(hv_tile_req),
                                cudaMemcpyHostToDevice, sl.st));
        HV_TRY(launch_render(L, (const hv_tile_req*)(sl.d_block + 16), n, mode, index, style, sl.d_out, sl.st));
    }
    HV_CUDA(cudaMemcpyAsync(sl.h_out, sl.d_out, (uint64_t)n * tb, cudaMemcpyDeviceToHost, sl.st));
    HV_CUDA(cudaEventRecord(sl.done, sl.st));
    return HV_OK;
}

// Can no object of the layer reach the tile?  Every sample lies inside the
// tile, so an object within R of one meets the tile's box widened by R, and
// a filled centre lies inside a polygon's box: both within the box of all the
// layer's objects (the R-tree's root box).
bool tile_unreachable(const Layer* L, const hv_tile_req& q) {
    const TreeView& v = L->tree.view;
    if (v.top == 0) return true;
    const int64_t span = (int64_t)1 << (31 - q.z);
    const int64_t X0 = -(int64_t)kGridHalf + (int64_t)q.x * span, Y0 = -(int64_t)kGridHalf + (int64_t)q.y * span;
    const int64_t R = (int64_t)q.r16 << (19 - q.z);
    const int4 b = v.root_box;
    return b.x > X0 + span + R || b.z < X0 - R || b.y > Y0 + span + R || b.w < Y0 - R;
}

void worker_main(Server* S) {
    cudaSetDevice(S->ctx->device);
    std::vector<int> to_launch, to_pool;
    while (true) {
        bool busy = false;
        to_launch.clear();
        to_pool.clear();
        {
            // look before locking: only this thread moves a slot into and out
            // of flight, so it may read those states without the lock; the lock
            // (which submitters and pollers share) is taken only when a batch
            // has completed or queued requests may find a free slot
            bool completed = false, in_flight = false, free_slot = false;
            for (auto& sl : S->slots) {
                const int st = __atomic_load_n(&sl.state, __ATOMIC_RELAXED);
                if (st == 0) free_slot = true;
                if (st != 1) continue;
                if (cudaEventQuery(sl.done) == cudaErrorNotReady)
                    in_flight = true;
                else
                    completed = true;
            }
            const bool waiting = __atomic_load_n(&S->queued, __ATOMIC_RELAXED) != 0;
            if (in_flight && !completed && !(waiting && free_slot)) {
                std::this_thread::yield();
                continue;
            }
        }
        {
            std::unique_lock<std::mutex> g(S->mu);
            // retire finished batches into the result pool
            for (size_t k = 0; k < S->slots.size(); k++) {
                Slot& sl = S->slots[k];
                if (sl.state != 1) continue;
                cudaError_t e = cudaEventQuery(sl.done);
                if (e == cudaErrorNotReady) { busy = true; continue; }
                double t = now_us();
                int st = e == cudaSuccess ? sl.status : HV_ECUDA;
                if (e != cudaSuccess) { S->error = cudaGetErrorString(e); cudaGetLastError(); }
                uint64_t tb = hv_tile_bytes(sl.items[0].req.mode);
                for (auto& it : sl.items)
                    S->done.push_back({it.tag, st, (uint32_t)tb, sl.h_out + it.offset, it.t_submit, sl.t_start, t,
                                       (int)k, nullptr});
                sl.outstanding = (int)sl.items.size();
                sl.state = 2;
                if (S->pool && st == HV_OK) to_pool.push_back((int)k);
            }
            // form batches for free slots: the oldest request's group, FIFO
            // within the group, while tile count and slot memory allow
            for (size_t k = 0; k < S->slots.size() && S->queued; k++) {
                Slot& sl = S->slots[k];
                if (sl.state != 0) continue;
                sl.items.clear();
                std::deque<Item>* grp = nullptr;
                for (auto& q : S->queues)
                    if (!q.second.empty() && (!grp || q.second.front().seq < grp->front().seq)) grp = &q.second;
                uint64_t tb = hv_tile_bytes(grp->front().req.mode);
                uint64_t used = 0;
                while (!grp->empty() && sl.items.size() < S->max_batch && used + tb <= S->slot_bytes) {
                    sl.items.push_back(grp->front());
                    grp->pop_front();
                    used += tb;
                    S->queued--;
                }
                sl.state = 1;
                sl.status = HV_OK;
                sl.t_start = now_us();
                to_launch.push_back((int)k);
            }
            if (S->stopping && S->queued == 0 && !busy && to_launch.empty() && to_pool.empty()) break;
            if (!busy && to_launch.empty() && to_pool.empty()) {
                S->cv.wait_for(g, std::chrono::microseconds(200));
                continue;
            }
        }
        // store the retired tiles in the result pool (only this thread
        // launches into a slot, so its tiles stay put meanwhile)
        for (int k : to_pool) {
            const Slot& sl = S->slots[k];
            const uint64_t tb = hv_tile_bytes(sl.items[0].req.mode);
            for (const auto& it : sl.items) pool_insert(S->pool, it.req, &S->opts.style, sl.h_out + it.offset, tb);
        }
        for (int k : to_launch) {
            int rc = launch_batch(S, k);
            std::lock_guard<std::mutex> g(S->mu);
            S->batches++;
            S->launched += S->slots[k].items.size();
            if (rc != HV_OK) {
                S->slots[k].status = rc;
                S->error = hv_last_error();
                cudaEventRecord(S->slots[k].done, S->slots[k].st);
            }
        }
        // batches in flight: poll their events again without sleeping (a
        // sleep's timer slack would add tens of microseconds to every batch)
        if (busy && to_launch.empty()) std::this_thread::yield();
    }
}

void destroy_server(Server* S) {
    cudaSetDevice(S->ctx->device);
    for (auto& sl : S->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        for (auto& g : sl.graphs) cudaGraphExecDestroy(g.second);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.h_block) cudaFreeHost(sl.h_block);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        dev_free(S->ctx, sl.d_block, 16 + (uint64_t)S->max_batch * sizeof(hv_tile_req));
        dev_free(S->ctx, sl.d_out, S->slot_bytes);
    }
    delete S;
}

}  // namespace
}  // namespace hv

using namespace hv;

extern "C" {

int hv_server_start(hv_ctx* ctx, hv_layer* const* layers, uint32_t n_layers, const hv_server_opts* opts,
                    hv_server** out) {
    if (!ctx || !out || (!layers && n_layers) || n_layers == 0) { set_error("hv_server_start: bad arguments"); return HV_EINVAL; }
    *out = nullptr;
    Ctx* c = (Ctx*)ctx;
    HV_CUDA(cudaSetDevice(c->device));
    Server* S = new Server();
    S->ctx = c;
    memset(&S->opts, 0, sizeof(S->opts));
    if (opts) S->opts = *opts;
    for (uint32_t i = 0; i < n_layers; i++) {
        Layer* L = (Layer*)layers[i];
        if (!L || L->ctx != c || !(L->indexes & HV_INDEX_RTREE)) {
            delete S;
            set_error("hv_server_start: layer %u is NULL, from another context, or not indexed", i);
            return HV_EINVAL;
        }
        S->layers.push_back(L);
    }
    S->pool = (ResultPool*)S->opts.pool;
    S->zeros.assign(hv_tile_bytes(HV_MODE_RGBA), 0);
    S->max_batch = S->opts.max_batch ? S->opts.max_batch : 64;
    if (S->max_batch > 4096) S->max_batch = 4096;
    if (!S->opts.queue_capacity) S->opts.queue_capacity = 65536;
    uint64_t scratch = S->opts.scratch_bytes ? S->opts.scratch_bytes : (1ull << 30);
    if (!S->opts.index_kind) S->opts.index_kind = HV_INDEX_RTREE;
    // a slot holds max_batch RGBA tiles; admission packs smaller tiles denser
    S->slot_bytes = (uint64_t)S->max_batch * hv_tile_bytes(HV_MODE_RGBA);
    uint64_t per_slot = S->slot_bytes + 16 + (uint64_t)S->max_batch * sizeof(hv_tile_req);
    uint64_t n_slots = scratch / per_slot;
    if (n_slots < 1) { delete S; set_error("hv_server_start: scratch_bytes holds no slot"); return HV_ENOMEM; }
    if (n_slots > 64) n_slots = 64;
    S->slots.resize(n_slots);
    for (auto& sl : S->slots) {
        int rc = HV_OK;
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void**)&sl.h_block, 16 + (uint64_t)S->max_batch * sizeof(hv_tile_req)) != cudaSuccess ||
            cudaMallocHost((void**)&sl.h_out, S->slot_bytes) != cudaSuccess)
            rc = HV_ECUDA;
        if (rc == HV_OK) rc = dev_alloc(c, (void**)&sl.d_block, 16 + (uint64_t)S->max_batch * sizeof(hv_tile_req));
        if (rc == HV_OK) rc = dev_alloc(c, (void**)&sl.d_out, S->slot_bytes);
        if (rc != HV_OK) {
            cudaGetLastError();
            destroy_server(S);
            if (rc == HV_ECUDA) set_error("hv_server_start: stream or pinned allocation failed");
            return rc;
        }
    }
    S->worker = std::thread(worker_main, S);
    *out = (hv_server*)S;
    return HV_OK;
}

int hv_server_submit(hv_server* srv, const hv_tile_req* req, uint64_t tag) {
    if (!srv || !req) { set_error("hv_server_submit: NULL argument"); return HV_EINVAL; }
    Server* S = (Server*)srv;
    const hv_tile_req& q = *req;
    if (q.layer >= S->layers.size() || hv_tile_bytes(q.mode) == 0) { set_error("hv_server_submit: bad layer or mode"); return HV_EINVAL; }
    if (q.z > 19 || q.x >= (1u << q.z) || q.y >= (1u << q.z) || q.r16 < 1 || q.r16 > 1024) {
        set_error("hv_server_submit: request out of range");
        return HV_ERANGE;
    }
    const double t = now_us();
    const uint32_t tb = (uint32_t)hv_tile_bytes(q.mode);
    // Parse Tasks: tiles the layer cannot reach, and tiles already in the pool
    std::shared_ptr<std::vector<uint8_t>> hit;
    const bool empty = tile_unreachable(S->layers[q.layer], q);
    if (!empty && S->pool) {
        auto v = std::make_shared<std::vector<uint8_t>>();
        if (pool_lookup(S->pool, q, &S->opts.style, v.get()) && v->size() == tb) hit = v;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stopping) { set_error("hv_server_submit: server is stopping"); return HV_ESTATE; }
    if (empty || hit) {
        S->done.push_back({tag, HV_OK, tb, hit ? hit->data() : S->zeros.data(), t, t, t, -1, hit});
        if (hit)
            S->pool_hits++;
        else
            S->empty_tiles++;
        return HV_OK;
    }
    if (S->queued >= S->opts.queue_capacity) { set_error("hv_server_submit: queue full"); return HV_EBUSY; }
    S->queues[((uint32_t)q.layer << 8) | q.mode].push_back({q, tag, t, S->seq++, 0});
    S->queued++;
    S->cv.notify_one();
    return HV_OK;
}

int hv_server_poll(hv_server* srv, hv_done* out, uint32_t max, uint32_t* n_out) {
    if (!srv || !n_out || (!out && max)) { set_error("hv_server_poll: NULL argument"); return HV_EINVAL; }
    Server* S = (Server*)srv;
    std::lock_guard<std::mutex> g(S->mu);
    // results handed out by the previous poll are no longer needed
    for (int k : S->exported) {
        Slot& sl = S->slots[k];
        if (sl.state == 3 && sl.outstanding == 0) sl.state = 0;
    }
    S->exported.clear();
    S->held.clear();
    uint32_t n = 0;
    while (n < max && !S->done.empty()) {
        Done d = S->done.front();
        S->done.pop_front();
        out[n].tag = d.tag;
        out[n].status = d.status;
        out[n].bytes = d.bytes;
        out[n].data = d.data;
        out[n].t_submit_us = d.t_submit;
        out[n].t_start_us = d.t_start;
        out[n].t_done_us = d.t_done;
        if (d.slot >= 0) {
            Slot& sl = S->slots[d.slot];
            if (--sl.outstanding == 0) {
                sl.state = 3;
                S->exported.push_back(d.slot);
            }
        } else if (d.own) {
            S->held.push_back(d.own);
        }
        n++;
    }
    *n_out = n;
    S->cv.notify_one();
    return HV_OK;
}

int hv_server_stop(hv_server* srv) {
    if (!srv) return HV_EINVAL;
    Server* S = (Server*)srv;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stopping = true;
        // unpolled results are dropped so their slots can drain
        S->done.clear();
        for (auto& sl : S->slots)
            if (sl.state >= 2) sl.state = 0;
        S->cv.notify_one();
    }
    // the worker exits once the queue is empty and no batch is in flight;
    // batches finish in bounded time, so wait with a generous limit
    auto t0 = std::chrono::steady_clock::now();
    while (true) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            bool in_flight = false;
            for (auto& sl : S->slots) in_flight |= sl.state == 1;
            // retired batches are recycled here, since nobody polls any more
            for (auto& sl : S->slots)
                if (sl.state >= 2) sl.state = 0;
            S->done.clear();
            if (S->queued == 0 && !in_flight) break;
        }
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(120)) {
            set_error("hv_server_stop: batches still in flight after 120 s");
            return HV_ETIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    S->worker.join();
    destroy_server(S);
    return HV_OK;
}

// Open-loop replay: submit reqs[i] at arrival_us[i] (relative to the call)
// from this thread, poll completions, and record each request's latency
// (done - arrival, microseconds) into latency_us[i] (tags are indices) and,
// if parts_us is given, its parts: parts_us[4i..4i+3] = wait before
// submission (the queue was full), task-pool wait (submission -> batch
// launch), service (launch -> completion seen by the worker: copies and
// kernels), hand-out (completion -> this thread's poll).
int hv_server_replay_detail(hv_server* srv, const hv_tile_req* reqs, const double* arrival_us, uint64_t n,
                            double* latency_us, double* parts_us, double* wall_us) {
    if (!srv || (n && (!reqs || !arrival_us || !latency_us)) || !wall_us) {
        set_error("hv_server_replay: NULL argument");
        return HV_EINVAL;
    }
    Server* S = (Server*)srv;
    std::vector<hv_done> buf(1024);
    uint64_t next = 0, finished = 0;
    double t0 = now_us();
    std::vector<double> submit_at(n, 0.0);
    while (finished < n) {
        double t = now_us() - t0;
        while (next < n && arrival_us[next] <= t) {
            int rc = hv_server_submit(srv, reqs + next, next);
            if (rc == HV_EBUSY) break;
            if (rc != HV_OK) return rc;
            submit_at[next] = t0 + arrival_us[next];
            next++;
        }
        uint32_t got = 0;
        HV_TRY(hv_server_poll(srv, buf.data(), (uint32_t)buf.size(), &got));
        for (uint32_t i = 0; i < got; i++) {
            if (buf[i].status != HV_OK) {
                set_error("hv_server_replay: request %llu failed (%d): %s", (unsigned long long)buf[i].tag,
                          buf[i].status, S->error.c_str());
                return buf[i].status;
            }
            const uint64_t k = buf[i].tag;
            const double polled = now_us();
            latency_us[k] = buf[i].t_done_us - submit_at[k];
            if (parts_us) {
                parts_us[4 * k] = buf[i].t_submit_us - submit_at[k];
                parts_us[4 * k + 1] = buf[i].t_start_us - buf[i].t_submit_us;
                parts_us[4 * k + 2] = buf[i].t_done_us - buf[i].t_start_us;
                parts_us[4 * k + 3] = polled - buf[i].t_done_us;
            }
            finished++;
        }
        if (got == 0) std::this_thread::yield();
    }
    *wall_us = now_us() - t0;
    return HV_OK;
}

int hv_server_replay(hv_server* srv, const hv_tile_req* reqs, const double* arrival_us, uint64_t n,
                     double* latency_us, double* wall_us) {
    return hv_server_replay_detail(srv, reqs, arrival_us, n, latency_us, nullptr, wall_us);
}

int hv_server_shortcuts(hv_server* srv, uint64_t* pool_hits, uint64_t* empty_tiles) {
    if (!srv) return HV_EINVAL;
    Server* S = (Server*)srv;
    std::lock_guard<std::mutex> g(S->mu);
    if (pool_hits) *pool_hits = S->pool_hits;
    if (empty_tiles) *empty_tiles = S->empty_tiles;
    return HV_OK;
}

int hv_server_stats(hv_server* srv, uint64_t* batches, uint64_t* tiles, uint64_t* graph_launches, uint32_t* slots) {
    if (!srv) return HV_EINVAL;
    Server* S = (Server*)srv;
    std::lock_guard<std::mutex> g(S->mu);
    if (batches) *batches = S->batches;
    if (tiles) *tiles = S->launched;
    if (graph_launches) *graph_launches = S->graph_launches;
    if (slots) *slots = (uint32_t)S->slots.size();
    return HV_OK;
}

}  // extern "C"
