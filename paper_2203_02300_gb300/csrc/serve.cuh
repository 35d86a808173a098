// Native serving runtime (the serving pattern of the batched matcher): several
// camera streams of different W x H x D submit frames from host memory; a
// scheduler thread admits pending frames into batches (a free device slot of
// the frame's stream, the batch's workspace within a lane's share of the
// memory budget), runs each batch on a free lane (a handle with its own
// workspace and CUDA stream: copies in, dco_stereo_match_batch, map copied
// straight into the caller's buffer), and one completion thread per lane
// retires that lane's batches on their events, waking the callers (a lane's
// batches finish in order on its stream; a short batch on one lane is never
// held up behind a long one on another).  Frames that
// arrive while other batches are on the device are admitted as slots and a
// lane free up, so their work overlaps on the device.  Included at the end
// of dco_stereo.cu; uses only the public C ABI for the matching itself.

#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvReq {
    int stream = 0, slot = -1;
    const uint8_t *left = nullptr, *right = nullptr;
    int16_t *out = nullptr;
    bool direct = false;   // all three buffers device-accessible: no staging copies
    unsigned long long ticket = 0;
    double arrival = 0, launch = 0, done = 0;
    float device_ms = 0;
    bool finished = false;
    dco_status status = DCO_OK;
};

struct SrvSlot {
    uint8_t *left = nullptr, *right = nullptr;
    int16_t *out = nullptr;
    bool busy = false;
};

struct SrvBatch {
    int lane = 0;
    bool hi = false;   // frames of latency-critical streams: the lane's high-priority stream
    cudaEvent_t start = nullptr, end = nullptr;
    std::vector<SrvReq *> reqs;
};

struct SrvLane {
    dco_stereo *h = nullptr;
    cudaStream_t stream = nullptr;      // batches of normal streams
    cudaStream_t stream_hi = nullptr;   // batches of latency-critical streams (greatest priority)
    bool busy = false;
    std::deque<SrvBatch> inflight;   // launched, not yet retired (at most one: the lane is busy meanwhile)
};

} // namespace

struct dco_server {
    int device = 0;
    dco_params params{};
    std::vector<dco_stream_desc> streams;
    std::vector<size_t> ws;                  // workspace bytes of one frame of each stream
    size_t lane_budget = 0;
    int max_batch = 16;
    std::vector<std::vector<SrvSlot>> slots;
    std::vector<SrvLane> lanes;
    std::mutex mu;
    std::condition_variable sched_cv, done_cv, wait_cv;
    std::deque<SrvReq *> pending;
    std::unordered_map<unsigned long long, SrvReq *> reqs;
    unsigned long long next_ticket = 1;
    bool stop = false;
    bool sched_done = false;                 // the scheduler has drained the pending frames and left
    std::thread sched;
    std::vector<std::thread> compl_;   // one completion thread per lane
    std::vector<cudaEvent_t> event_pool;
    unsigned long long batches = 0, frames_batched = 0;
    size_t max_batch_bytes = 0;
};

namespace {

size_t stream_ws(const dco_params &p, const dco_stream_desc &d)
{
    dco_params q = p;
    if (d.d_chunk > 0) q.d_chunk = d.d_chunk;
    return dco_stereo_workspace_bytes(d.W, d.H, d.D, &q);
}

cudaEvent_t srv_event(dco_server *s)
{
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// a pending frame of stream `st` can be admitted now (a free slot)
bool srv_slot_free(const dco_server *s, int st)
{
    for (const SrvSlot &sl : s->slots[st])
        if (!sl.busy) return true;
    return false;
}

// The next batch: frames of latency-critical streams first (a batch holds
// frames of one class only), in arrival order within the class, while the
// batch has room, the frame's stream has a free slot and the lane's share
// of the budget holds its workspace; the frames left behind keep their
// order.  Caller holds mu.
std::vector<SrvReq *> srv_form_batch(dco_server *s, bool &hi)
{
    std::vector<SrvReq *> batch;
    std::deque<SrvReq *> skipped;
    size_t used = 0;
    hi = false;
    for (const SrvReq *r : s->pending)
        if (s->streams[r->stream].priority && srv_slot_free(s, r->stream)) {
            hi = true;
            break;
        }
    while (!s->pending.empty() && (int)batch.size() < s->max_batch) {
        SrvReq *r = s->pending.front();
        s->pending.pop_front();
        int si = -1;
        for (size_t k = 0; k < s->slots[r->stream].size(); k++)
            if (!s->slots[r->stream][k].busy) {
                si = (int)k;
                break;
            }
        if (si < 0 || (s->streams[r->stream].priority != 0) != hi || used + s->ws[r->stream] > s->lane_budget) {
            skipped.push_back(r);
            continue;
        }
        r->slot = si;
        s->slots[r->stream][si].busy = true;
        used += s->ws[r->stream];
        batch.push_back(r);
    }
    s->max_batch_bytes = std::max(s->max_batch_bytes, used);
    while (!skipped.empty()) {
        s->pending.push_front(skipped.back());
        skipped.pop_back();
    }
    return batch;
}

// copies in, the batched match, the maps out, on the lane's stream of the
// batch's class
dco_status srv_launch(dco_server *s, SrvLane &ln, const std::vector<SrvReq *> &batch, SrvBatch &b)
{
    cudaSetDevice(s->device);
    (void)cudaGetLastError();
    std::vector<dco_pair_desc> descs(batch.size());
    const cudaStream_t cs = b.hi ? ln.stream_hi : ln.stream;
    if (cudaEventRecord(b.start, cs) != cudaSuccess) return DCO_ECUDA;
    for (size_t k = 0; k < batch.size(); k++) {
        const SrvReq *r = batch[k];
        const dco_stream_desc &d = s->streams[r->stream];
        const SrvSlot &sl = s->slots[r->stream][r->slot];
        if (r->direct) {   // the device reads the images and writes the map in place
            descs[k] = dco_pair_desc{r->left, r->right, d.W, d.H, d.D, r->out, d.d_chunk, d.h_chunk, d.v_chunk};
            continue;
        }
        const size_t img = (size_t)d.W * d.H * 3;
        if (cudaMemcpyAsync(sl.left, r->left, img, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
            cudaMemcpyAsync(sl.right, r->right, img, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            return DCO_ECUDA;
        descs[k] = dco_pair_desc{sl.left, sl.right, d.W, d.H, d.D, sl.out, d.d_chunk, d.h_chunk, d.v_chunk};
    }
    dco_status st = dco_stereo_match_batch(ln.h, descs.data(), (int)descs.size(), &s->params, cs);
    if (st != DCO_OK) return st;
    for (const SrvReq *r : batch) {
        if (r->direct) continue;
        const dco_stream_desc &d = s->streams[r->stream];
        const SrvSlot &sl = s->slots[r->stream][r->slot];
        if (cudaMemcpyAsync(r->out, sl.out, (size_t)d.W * d.H * 2, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
            return DCO_ECUDA;
    }
    return cudaEventRecord(b.end, cs) == cudaSuccess ? DCO_OK : DCO_ECUDA;
}

void srv_schedule(dco_server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        int li = -1;
        s->sched_cv.wait(lk, [&] {
            li = -1;
            for (size_t k = 0; k < s->lanes.size(); k++)
                if (!s->lanes[k].busy) li = (int)k;
            return (s->stop && s->pending.empty()) || (!s->pending.empty() && li >= 0);
        });
        if (s->pending.empty()) break;   // stopping, nothing left to admit
        bool hi = false;
        std::vector<SrvReq *> batch = srv_form_batch(s, hi);
        if (batch.empty()) {   // every pending frame waits for a slot: wait for a completion
            s->sched_cv.wait_for(lk, std::chrono::milliseconds(1));
            continue;
        }
        SrvLane &ln = s->lanes[li];
        ln.busy = true;
        SrvBatch b;
        b.lane = li;
        b.hi = hi;
        b.start = srv_event(s);
        b.end = srv_event(s);
        b.reqs = batch;
        const double t = now_s();
        for (SrvReq *r : batch) r->launch = t;
        lk.unlock();
        const dco_status st = srv_launch(s, ln, batch, b);
        lk.lock();
        if (st != DCO_OK) {   // this batch's requests fail; the server keeps serving
            cudaStreamSynchronize(hi ? ln.stream_hi : ln.stream);
            (void)cudaGetLastError();
            for (SrvReq *r : batch) {
                r->status = st;
                r->finished = true;
                r->done = now_s();
                s->slots[r->stream][r->slot].busy = false;
            }
            ln.busy = false;
            s->event_pool.push_back(b.start);
            s->event_pool.push_back(b.end);
            s->wait_cv.notify_all();
            continue;
        }
        s->batches++;
        s->frames_batched += batch.size();
        ln.inflight.push_back(b);
        s->done_cv.notify_all();
    }
    s->sched_done = true;
    s->done_cv.notify_all();
}

void srv_complete(dco_server *s, int lane)
{
    cudaSetDevice(s->device);
    SrvLane &ln = s->lanes[lane];
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->done_cv.wait(lk, [&] { return !ln.inflight.empty() || s->sched_done; });
        if (ln.inflight.empty()) break;   // the scheduler has left and this lane's batches are retired
        SrvBatch b = ln.inflight.front();
        ln.inflight.pop_front();
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(b.end);
        const double t = now_s();
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, b.start, b.end);
        lk.lock();
        for (SrvReq *r : b.reqs) {
            r->done = t;
            r->device_ms = ms;
            r->status = e == cudaSuccess ? DCO_OK : DCO_ECUDA;
            r->finished = true;
            s->slots[r->stream][r->slot].busy = false;
        }
        s->lanes[b.lane].busy = false;
        s->event_pool.push_back(b.start);
        s->event_pool.push_back(b.end);
        s->wait_cv.notify_all();
        s->sched_cv.notify_all();
    }
}

void srv_free(dco_server *s)
{
    cudaSetDevice(s->device);
    for (auto &ln : s->lanes) {
        if (ln.stream) cudaStreamSynchronize(ln.stream);
        if (ln.stream_hi) cudaStreamSynchronize(ln.stream_hi);
        dco_stereo_destroy(ln.h);
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.stream_hi) cudaStreamDestroy(ln.stream_hi);
    }
    for (auto &v : s->slots)
        for (auto &sl : v) {
            cudaFree(sl.left);
            cudaFree(sl.right);
            cudaFree(sl.out);
        }
    for (auto e : s->event_pool) cudaEventDestroy(e);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
}

} // namespace

extern "C" {

dco_status dco_server_create(dco_server **out, int device, const dco_stream_desc *streams, int nstreams, int lanes,
                             int slots_per_stream, int max_batch, size_t budget_bytes, const dco_params *pin)
{
    if (!out) return DCO_EINVAL;
    *out = nullptr;
    if (!streams || nstreams < 1 || lanes < 1 || lanes > 16 || slots_per_stream < 1 || max_batch < 1)
        return DCO_EINVAL;
    dco_params p;
    if (pin) p = *pin;
    else dco_params_default(&p);
    if (!params_valid(p)) return DCO_EINVAL;
    for (int i = 0; i < nstreams; i++)
        if (!dims_valid(streams[i].W, streams[i].H, streams[i].D, p.d_min) || streams[i].d_chunk < 0 ||
            !tile_valid(streams[i].h_chunk) || !tile_valid(streams[i].v_chunk) ||
            (streams[i].priority != 0 && streams[i].priority != 1))
            return DCO_EINVAL;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DCO_EINVAL;
    dco_server *s = new (std::nothrow) dco_server();
    if (!s) return DCO_ENOMEM;
    s->device = device;
    s->params = p;
    s->max_batch = max_batch;
    s->streams.assign(streams, streams + nstreams);
    size_t total = 0, largest = 0;
    for (const auto &d : s->streams) {
        s->ws.push_back(stream_ws(p, d));
        total += s->ws.back();
        largest = std::max(largest, s->ws.back());
    }
    // default budget: every stream's frame can be in every lane's batch
    if (!budget_bytes) budget_bytes = (size_t)lanes * total;
    s->lane_budget = budget_bytes / lanes;
    if (largest > s->lane_budget) {
        delete s;
        return DCO_EBUDGET;   // a lane could not hold one frame of the largest stream
    }
    cudaSetDevice(device);
    dco_status st = DCO_OK;
    s->slots.resize(nstreams);
    for (int i = 0; i < nstreams && st == DCO_OK; i++) {
        const dco_stream_desc &d = s->streams[i];
        s->slots[i].resize(slots_per_stream);
        for (auto &sl : s->slots[i]) {
            const size_t img = (size_t)d.W * d.H * 3;
            if (cudaMalloc((void **)&sl.left, img) != cudaSuccess || cudaMalloc((void **)&sl.right, img) != cudaSuccess ||
                cudaMalloc((void **)&sl.out, (size_t)d.W * d.H * 2) != cudaSuccess ||
                cudaMemset(sl.left, 0, img) != cudaSuccess || cudaMemset(sl.right, 0, img) != cudaSuccess) {
                st = DCO_ENOMEM;
                break;
            }
        }
    }
    s->lanes.resize(lanes);
    for (auto &ln : s->lanes) {
        if (st != DCO_OK) break;
        if ((st = dco_stereo_create(&ln.h, device, s->lane_budget)) != DCO_OK) break;
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&ln.stream, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&ln.stream_hi, cudaStreamNonBlocking, greatest) != cudaSuccess)
            st = DCO_ECUDA;
    }
    // warm every lane up with the largest batch admission allows, so its
    // workspace never grows (a synchronising reallocation) while serving
    if (st == DCO_OK) {
        std::vector<dco_pair_desc> warm;
        size_t used = 0;
        for (int i = 0; i < nstreams; i++)
            for (auto &sl : s->slots[i]) {
                const dco_stream_desc &d = s->streams[i];
                if (used + s->ws[i] <= s->lane_budget && (int)warm.size() < max_batch) {
                    warm.push_back(dco_pair_desc{sl.left, sl.right, d.W, d.H, d.D, sl.out, d.d_chunk, d.h_chunk, d.v_chunk});
                    used += s->ws[i];
                }
            }
        for (auto &ln : s->lanes) {
            if ((st = dco_stereo_match_batch(ln.h, warm.data(), (int)warm.size(), &p, ln.stream)) != DCO_OK) break;
            if (cudaStreamSynchronize(ln.stream) != cudaSuccess) {
                st = DCO_ECUDA;
                break;
            }
        }
    }
    if (st != DCO_OK) {
        srv_free(s);
        return st;
    }
    s->sched = std::thread(srv_schedule, s);
    for (int k = 0; k < (int)s->lanes.size(); k++) s->compl_.emplace_back(srv_complete, s, k);
    *out = s;
    return DCO_OK;
}

dco_status dco_server_submit(dco_server *s, int stream, const uint8_t *left, const uint8_t *right,
                             int16_t *disp_out, unsigned long long *ticket)
{
    if (!s || !left || !right || !disp_out || !ticket || stream < 0 || stream >= (int)s->streams.size())
        return DCO_EINVAL;
    SrvReq *r = new (std::nothrow) SrvReq();
    if (!r) return DCO_ENOMEM;
    r->stream = stream;
    r->left = left;
    r->right = right;
    r->out = disp_out;
    // pinned, registered or managed host buffers are read and written by the
    // kernels in place (over NVLink-C2C on Grace systems), as in
    // dco_stereo_match_host; other buffers go through the stream's device slots
    r->direct = s->params.vote_iters == 0 && device_accessible(left) && device_accessible(right) &&
                device_accessible(disp_out);
    r->arrival = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return DCO_EINVAL;
        }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->pending.push_back(r);
    }
    *ticket = r->ticket;
    s->sched_cv.notify_all();
    return DCO_OK;
}

dco_status dco_server_wait(dco_server *s, unsigned long long ticket, int timeout_ms, dco_request_times *times)
{
    if (!s) return DCO_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return DCO_EINVAL;
    SrvReq *r = it->second;
    if (timeout_ms < 0) s->wait_cv.wait(lk, [&] { return r->finished; });
    else if (!s->wait_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->finished; }))
        return DCO_ETIMEOUT;
    if (times) {
        times->arrival_s = r->arrival;
        times->launch_s = r->launch;
        times->done_s = r->done;
        times->device_ms = r->device_ms;
    }
    const dco_status st = r->status;
    s->reqs.erase(it);
    delete r;
    return st;
}

dco_status dco_server_counters(dco_server *s, unsigned long long *batches, unsigned long long *frames,
                               size_t *max_batch_bytes, size_t *lane_budget)
{
    if (!s) return DCO_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (batches) *batches = s->batches;
    if (frames) *frames = s->frames_batched;
    if (max_batch_bytes) *max_batch_bytes = s->max_batch_bytes;
    if (lane_budget) *lane_budget = s->lane_budget;
    return DCO_OK;
}

void dco_server_destroy(dco_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->sched_cv.notify_all();
    s->sched.join();   // admits and launches every pending frame first
    for (auto &t : s->compl_) t.join();   // then every batch in flight is retired
    srv_free(s);
}

} // extern "C"
