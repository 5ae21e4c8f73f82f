// Serving runtime of libspx (spx_server_* in include/spx.h): a thread that
// batches queued requests, runs each batch's count pass, admits its outputs
// against a device-memory budget, runs the write pass (and, for selections,
// the partition into per-query lists) and timestamps completion from a stream
// callback.  All device work is in kernels.cu; this file only schedules it.
#include "kernels.h"
#include "server_internal.h"
#include "spx.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace spx;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    spx_request rq{};
    uint32_t P = 0;
    int status = SPX_EBUSY;
    uint32_t batch_size = 0;
    double t_submit = 0, t_start = 0, t_counted = 0, t_written = 0, t_done = 0;
    uint64_t total = 0;
    // outputs (kept until released): join pairs | selection ids + offsets
    void *out_mem = nullptr;
    size_t out_bytes = 0;
    unsigned long long *counts = nullptr; // join: allocated when the batch starts
    size_t counts_bytes = 0;
    // selection temporaries: pairs in point order + partition scratch
    void *tmp_mem = nullptr;
    size_t tmp_bytes = 0;
    // per-request passes: the join's scratch (per-point results, chunk
    // offsets) from the count pass to the write pass
    void *join_mem = nullptr;
    size_t join_bytes = 0;
    // a request that brought its own polygons: their host copy, and the index
    // built on the device when its batch starts (from the pool, freed after
    // its write pass)
    bool own = false;
    std::vector<int32_t> xy;
    std::vector<uint64_t> off;
    IndexView own_view{};
    void *own_mem = nullptr;
    size_t own_bytes = 0;
    int readers = 0; // spx_server_read calls copying the outputs (release waits for none)
};

struct Slot {
    enum State { kIdle, kCounting, kAdmit, kEmitting };
    cudaStream_t s = nullptr;
    void *scratch = nullptr;
    unsigned long long *dev_words = nullptr;  // kMaxBatch totals | error word | stats
    unsigned long long *host_words = nullptr; // pinned copy of totals | error word
    std::vector<Req *> batch;
    State state = kIdle;
    bool waited = false;             // the current batch has waited for budget
    std::atomic<int> flag{0};        // set by the stream callbacks: 1 counted, 2 written
    std::atomic<double> t_cb{0.0};   // callback time (ms)
    struct spx_server *srv = nullptr;
};

constexpr int kWordErr = kMaxBatch;       // error word position in dev_words / host_words
constexpr int kWordStats = kMaxBatch + 1; // kStatCount counters

} // namespace

struct spx_server {
    ServedData data;
    spx_server_params prm{};
    int max_batch = kMaxBatch;
    Clock::time_point t0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t release_stream = nullptr;
    std::vector<std::unique_ptr<Slot>> slots;
    std::thread worker;
    std::mutex mu;                   // server state (the worker holds it across CUDA calls)
    std::mutex cv_mu;                // wake-ups only: never held across a CUDA call
    std::condition_variable cv;      // wakes the worker (with cv_mu)
    std::condition_variable cv_done; // wakes waiters
    std::deque<Req *> queue;
    std::map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_id = 1;
    bool stopping = false;
    uint64_t used = 0;
    spx_server_stats_t st{};
    std::string err;
    std::atomic<int> events{0};

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
    // count an event that may let the worker progress and wake it
    void signal()
    {
        {
            std::lock_guard<std::mutex> lk(cv_mu);
            events.fetch_add(1);
        }
        cv.notify_all();
    }
    const IndexView &view_of(const Req *r) const { return r->own ? r->own_view : data.ix[r->rq.index]; }
    int fp32_of(const Req *r) const { return r->own ? 1 : data.fp32[r->rq.index]; }
    void retire_own(Req *r, cudaStream_t s);
    bool build_own(Slot &sl);
    void run();
    bool start_batch(Slot &sl);
    JoinLaunch request_launch(Slot &sl, const Req *r, size_t i) const;
    void counted(Slot &sl);
    bool admit(Slot &sl);
    void written(Slot &sl);
    void fail_batch(Slot &sl, int status);
};

namespace {

void CUDART_CB on_stream_point(void *p)
{
    // Runs on CUDA's host-function thread: no CUDA calls here, and never the
    // server mutex -- the worker holds that across CUDA calls, some of which
    // (lazy module loading on a kernel's first launch, for one) can wait for
    // pending host functions.  The slot's flag is atomic; the wake-up goes
    // through cv_mu, which nobody holds across a CUDA call.
    Slot *sl = static_cast<Slot *>(p);
    spx_server *srv = sl->srv;
    sl->t_cb.store(srv->now_ms());
    sl->flag.fetch_add(1);
    srv->signal();
}

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

bool pool_alloc(spx_server *srv, void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (!bytes)
        return true;
    return cudaMallocFromPoolAsync(p, bytes, srv->pool, s) == cudaSuccess;
}

void pool_free(void *p, cudaStream_t s)
{
    if (p)
        cudaFreeAsync(p, s);
}

} // namespace

void spx_server::fail_batch(Slot &sl, int status)
{
    for (Req *r : sl.batch) {
        retire_own(r, sl.s);
        pool_free(r->out_mem, sl.s);
        pool_free(r->tmp_mem, sl.s);
        pool_free(r->counts, sl.s);
        pool_free(r->join_mem, sl.s);
        used -= r->out_bytes + r->tmp_bytes + r->counts_bytes + r->join_bytes;
        r->out_mem = r->tmp_mem = r->join_mem = nullptr;
        r->counts = nullptr;
        r->out_bytes = r->tmp_bytes = r->counts_bytes = r->join_bytes = 0;
        r->status = status;
        r->t_done = now_ms();
        st.failed++;
    }
    sl.batch.clear();
    sl.state = Slot::kIdle;
    cv_done.notify_all();
}

// A finished request's own index back to the pool, after its batch's work on s.
void spx_server::retire_own(Req *r, cudaStream_t s)
{
    pool_free(r->own_mem, s);
    used -= r->own_bytes;
    r->own_mem = nullptr;
    r->own_bytes = 0;
}

// Indexes of the batch's requests that brought their polygons, built on the
// device now, on the slot's stream with memory from the pool (the worker waits
// on that stream alone; the build counts in the request's latency).  False:
// the batch failed.
bool spx_server::build_own(Slot &sl)
{
    for (Req *r : sl.batch) {
        if (!r->own || r->own_mem)
            continue;
        std::string why;
        const int b = device_grid_index(r->xy.data(), r->off.data(), r->P, r->own_view, r->own_mem, r->own_bytes, why,
                                        sl.s, pool);
        if (b != 0) {
            err = "server: device build of a request's polygon index failed: " + why;
            fail_batch(sl, b == 1 ? SPX_EINVAL : SPX_ECUDA);
            return false;
        }
        used += r->own_bytes;
        st.peak_bytes_in_use = std::max(st.peak_bytes_in_use, used);
    }
    return true;
}

// The join launch of request r, position i of its slot's batch (outputs and
// capacity are set by the write pass).
JoinLaunch spx_server::request_launch(Slot &sl, const Req *r, size_t i) const
{
    JoinLaunch a{};
    a.ix = view_of(r);
    a.ix.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
    a.pts = data.pts;
    a.n = data.n;
    a.counts = r->counts;
    a.total = sl.dev_words + i;
    a.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
    a.stats = sl.dev_words + kWordStats;
    a.fp32 = fp32_of(r);
    return a;
}

// Take the waiting requests (arrival order) into a batch and launch its count
// pass.  False: nothing started (the per-request join scratch does not fit the
// budget while other batches hold memory; a release wakes the worker).
bool spx_server::start_batch(Slot &sl)
{
    if (!prm.plain && !prm.fused) {
        const uint64_t per = up256(join_scratch_bytes(data.n));
        const uint64_t k = std::min<uint64_t>(queue.size(), uint64_t(max_batch));
        if (used > 0 && used + k * per > prm.output_budget && !stopping) {
            if (!sl.waited)
                st.admission_waits++;
            sl.waited = true;
            return false;
        }
        sl.waited = false;
    }
    sl.batch.clear();
    uint32_t hist = 0;
    while (!queue.empty() && (int)sl.batch.size() < max_batch) {
        Req *r = queue.front();
        const uint32_t h = r->rq.kind == SPX_REQ_JOIN ? r->P : 0u;
        if (prm.fused && !sl.batch.empty() && hist + h > kMultiHistMax)
            break; // keep the fused pass's per-polygon counters in shared memory
        hist += h;
        sl.batch.push_back(r);
        queue.pop_front();
    }
    const double t = now_ms();
    const uint32_t K = uint32_t(sl.batch.size());
    for (Req *r : sl.batch) {
        r->t_start = t;
        r->batch_size = K;
    }
    if (!build_own(sl))
        return true;
    st.batches++;
    st.batched_requests += K;
    // join counts are produced by the count pass (batched) or the write pass (plain)
    for (Req *r : sl.batch)
        if (r->rq.kind == SPX_REQ_JOIN) {
            r->counts_bytes = up256(size_t(std::max(r->P, 1u)) * 8);
            void *p = nullptr;
            if (!pool_alloc(this, &p, r->counts_bytes, sl.s)) {
                r->counts_bytes = 0;
                err = "server: allocation of join counts failed";
                fail_batch(sl, SPX_ENOMEM);
                return true;
            }
            r->counts = static_cast<unsigned long long *>(p);
            used += r->counts_bytes;
        }
    st.peak_bytes_in_use = std::max(st.peak_bytes_in_use, used);
    cudaError_t e = cudaSuccess;
    if (prm.plain) {
        Req *r = sl.batch[0];
        JoinLaunch a{};
        a.ix = view_of(r);
        a.ix.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
        a.pts = data.pts;
        a.n = data.n;
        a.counts = r->counts;
        a.total = sl.dev_words;
        a.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
        a.stats = sl.dev_words + kWordStats;
        a.fp32 = 0;
        e = launch_plain_count(a, sl.scratch, sl.s);
    } else if (!prm.fused) {
        // each request through the join's own passes 1 and 2, its results
        // kept in its scratch until the write pass
        for (uint32_t i = 0; i < K && e == cudaSuccess; ++i) {
            Req *r = sl.batch[i];
            r->join_bytes = up256(join_scratch_bytes(data.n));
            if (!pool_alloc(this, &r->join_mem, r->join_bytes, sl.s)) {
                r->join_bytes = 0;
                err = "server: allocation of join scratch failed";
                fail_batch(sl, SPX_ENOMEM);
                return true;
            }
            used += r->join_bytes;
            e = launch_join_count(request_launch(sl, r, i), r->join_mem, sl.s);
        }
        st.peak_bytes_in_use = std::max(st.peak_bytes_in_use, used);
    } else {
        MultiLaunch m{};
        m.K = int(K);
        m.pts = data.pts;
        m.n = data.n;
        m.fp32 = 1;
        m.totals = sl.dev_words;
        m.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
        m.stats = sl.dev_words + kWordStats;
        m.qbase[0] = 0;
        for (uint32_t i = 0; i < K; ++i) {
            const Req *r = sl.batch[i];
            m.ix[i] = view_of(r);
            m.ix[i].err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
            m.fp32 &= fp32_of(r);
            m.counts[i] = r->counts;
            m.qbase[i + 1] = m.qbase[i] + (r->counts ? r->P : 0u);
        }
        e = launch_multi_count(m, sl.scratch, sl.s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.host_words, sl.dev_words, sizeof(unsigned long long) * (kMaxBatch + 1),
                            cudaMemcpyDeviceToHost, sl.s);
    if (e == cudaSuccess)
        e = cudaLaunchHostFunc(sl.s, on_stream_point, &sl);
    if (e != cudaSuccess) {
        err = std::string("server: count pass launch failed: ") + cudaGetErrorString(e);
        fail_batch(sl, SPX_ECUDA);
        return true;
    }
    sl.state = Slot::kCounting;
    return true;
}

// Count pass done: sizes of every output.
void spx_server::counted(Slot &sl)
{
    if (sl.host_words[kWordErr]) {
        err = "server: a kernel reported an error in the count pass";
        cudaMemsetAsync(sl.dev_words + kWordErr, 0, 8, sl.s);
        fail_batch(sl, SPX_EKERNEL);
        return;
    }
    const double t = sl.t_cb.load();
    for (size_t i = 0; i < sl.batch.size(); ++i) {
        Req *r = sl.batch[i];
        r->t_counted = t;
        r->total = sl.host_words[i];
        if (r->rq.kind == SPX_REQ_JOIN) {
            r->out_bytes = up256(std::max<uint64_t>(r->total, 1) * 8);
        } else {
            r->out_bytes = up256(std::max<uint64_t>(r->total, 1) * 4) + up256(size_t(r->P + 1) * 8);
            r->tmp_bytes = up256(std::max<uint64_t>(r->total, 1) * 8) + up256(partition_scratch_bytes(r->total, r->P));
        }
    }
    sl.state = Slot::kAdmit;
}

// Allocate the outputs if the budget allows and launch the write pass.
bool spx_server::admit(Slot &sl)
{
    uint64_t need = 0;
    for (Req *r : sl.batch)
        need += r->out_bytes + r->tmp_bytes;
    // bytes held by anything but the batches waiting here (their join counters
    // and scratch must not keep each other out)
    uint64_t waiting = 0;
    for (auto &o : slots)
        if (o->state == Slot::kAdmit)
            for (Req *r : o->batch)
                waiting += r->counts_bytes + r->join_bytes;
    const uint64_t other = used - waiting;
    if (used + need > prm.output_budget && other > 0 && !stopping) {
        // wait for releases (a batch that fits no budget runs once nothing else is held)
        if (!sl.waited)
            st.admission_waits++;
        sl.waited = true;
        return false;
    }
    sl.waited = false;
    for (Req *r : sl.batch) {
        if (!pool_alloc(this, &r->out_mem, r->out_bytes, sl.s) || !pool_alloc(this, &r->tmp_mem, r->tmp_bytes, sl.s)) {
            for (Req *q : sl.batch) {
                if (q->out_mem) {
                    pool_free(q->out_mem, sl.s);
                    q->out_mem = nullptr;
                }
                if (q->tmp_mem) {
                    pool_free(q->tmp_mem, sl.s);
                    q->tmp_mem = nullptr;
                }
                q->out_bytes = q->tmp_bytes = 0;
            }
            err = "server: output allocation failed";
            fail_batch(sl, SPX_ENOMEM);
            return true;
        }
    }
    used += need;
    st.peak_bytes_in_use = std::max(st.peak_bytes_in_use, used);
    cudaError_t e = cudaSuccess;
    // write targets: join pairs straight into the output; selection pairs into the temporary
    auto pairs_of = [](Req *r) {
        return static_cast<uint2 *>(r->rq.kind == SPX_REQ_JOIN ? r->out_mem : r->tmp_mem);
    };
    if (prm.plain) {
        Req *r = sl.batch[0];
        JoinLaunch a{};
        a.ix = view_of(r);
        a.ix.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
        a.pts = data.pts;
        a.n = data.n;
        a.pairs = pairs_of(r);
        a.cap = r->total;
        a.counts = r->counts;
        a.total = sl.dev_words;
        a.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
        a.stats = sl.dev_words + kWordStats;
        e = launch_plain_write(a, sl.scratch, sl.s);
    } else if (!prm.fused) {
        for (size_t i = 0; i < sl.batch.size() && e == cudaSuccess; ++i) {
            Req *r = sl.batch[i];
            JoinLaunch a = request_launch(sl, r, i);
            a.pairs = pairs_of(r);
            a.cap = r->total;
            e = launch_join_write(a, r->join_mem, sl.s);
        }
    } else {
        MultiLaunch m{};
        m.K = int(sl.batch.size());
        m.pts = data.pts;
        m.n = data.n;
        m.fp32 = 1;
        m.totals = sl.dev_words;
        m.err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
        m.stats = sl.dev_words + kWordStats;
        for (int i = 0; i < m.K; ++i) {
            Req *r = sl.batch[i];
            m.ix[i] = view_of(r);
            m.ix[i].err = reinterpret_cast<unsigned *>(sl.dev_words + kWordErr);
            m.fp32 &= fp32_of(r);
            m.pairs[i] = pairs_of(r);
            m.cap[i] = r->total;
        }
        e = launch_multi_emit(m, sl.scratch, sl.s);
    }
    for (size_t i = 0; i < sl.batch.size() && e == cudaSuccess; ++i) {
        Req *r = sl.batch[i];
        if (r->rq.kind != SPX_REQ_SELECT)
            continue;
        char *o = static_cast<char *>(r->out_mem);
        uint32_t *ids = reinterpret_cast<uint32_t *>(o);
        unsigned long long *offs =
            reinterpret_cast<unsigned long long *>(o + up256(std::max<uint64_t>(r->total, 1) * 4));
        char *t = static_cast<char *>(r->tmp_mem);
        void *part = t + up256(std::max<uint64_t>(r->total, 1) * 8);
        e = launch_partition(reinterpret_cast<const uint2 *>(t), sl.dev_words + i, r->total, r->P, ids, offs, part,
                             sl.s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.host_words + kWordErr, sl.dev_words + kWordErr, 8, cudaMemcpyDeviceToHost, sl.s);
    if (e == cudaSuccess)
        e = cudaLaunchHostFunc(sl.s, on_stream_point, &sl);
    if (e != cudaSuccess) {
        err = std::string("server: write pass launch failed: ") + cudaGetErrorString(e);
        fail_batch(sl, SPX_ECUDA);
        return true;
    }
    const double t = now_ms();
    for (Req *r : sl.batch)
        r->t_written = t;
    sl.state = Slot::kEmitting;
    return true;
}

// Write pass done: results are complete.
void spx_server::written(Slot &sl)
{
    const double t = sl.t_cb.load();
    const bool bad = sl.host_words[kWordErr] != 0;
    if (bad) {
        err = "server: a kernel reported an error in the write pass";
        cudaMemsetAsync(sl.dev_words + kWordErr, 0, 8, sl.s);
        fail_batch(sl, SPX_EKERNEL);
        return;
    }
    for (Req *r : sl.batch) {
        retire_own(r, sl.s);
        pool_free(r->tmp_mem, sl.s); // ordered after the partition on this stream
        pool_free(r->join_mem, sl.s);
        r->tmp_mem = r->join_mem = nullptr;
        used -= r->tmp_bytes + r->join_bytes;
        r->tmp_bytes = r->join_bytes = 0;
        r->t_done = t;
        r->status = SPX_OK;
        st.completed++;
    }
    sl.batch.clear();
    sl.state = Slot::kIdle;
    cv_done.notify_all();
}

void spx_server::run()
{
    cudaSetDevice(data.device);
    for (;;) {
        // events seen before this pass: any later one ends the wait below
        const int ev0 = events.load();
        std::unique_lock<std::mutex> lk(mu);
        bool progress = false;
        for (auto &up : slots) {
            Slot &sl = *up;
            if (sl.state == Slot::kCounting && sl.flag.load() >= 1) {
                counted(sl);
                progress = true;
            }
            if (sl.state == Slot::kAdmit && admit(sl))
                progress = true;
            if (sl.state == Slot::kEmitting && sl.flag.load() >= 2) {
                sl.flag.store(0);
                written(sl);
                progress = true;
            }
            if (sl.state == Slot::kIdle && !queue.empty()) {
                sl.flag.store(0);
                if (start_batch(sl))
                    progress = true;
            }
        }
        if (stopping && queue.empty()) {
            bool idle = true;
            for (auto &up : slots)
                idle = idle && up->state == Slot::kIdle;
            if (idle)
                break;
        }
        lk.unlock();
        if (!progress) {
            std::unique_lock<std::mutex> lw(cv_mu);
            cv.wait_for(lw, std::chrono::milliseconds(50), [&] { return events.load() != ev0; });
        }
    }
}

extern "C" {

spx_status spx_server_create(spx_ctx *ctx, spx_points points, const spx_index *indexes, uint32_t n_indexes,
                             const spx_server_params *params, spx_server **out)
{
    if (!ctx || !out || (n_indexes && !indexes))
        return SPX_EINVAL;
    *out = nullptr;
    spx_server_params prm{};
    if (params) {
        prm = *params;

        for (int r : prm.reserved)
            if (r)
                return ctx_error(ctx, SPX_EINVAL, "server: reserved fields must be zero");
    }
    if (prm.max_batch == 0)
        prm.max_batch = kMaxBatch;
    if (prm.slots == 0)
        prm.slots = 2;
    if (prm.max_batch < 1 || prm.max_batch > kMaxBatch || prm.slots < 1 || prm.slots > 4 ||
        (prm.plain != 0 && prm.plain != 1) || (prm.fused != 0 && prm.fused != 1))
        return ctx_error(ctx, SPX_EINVAL,
                         "server: need 1 <= max_batch <= 8, 1 <= slots <= 4, plain and fused 0 or 1");
    if (prm.plain)
        prm.max_batch = prm.slots = 1;
    auto srv = std::make_unique<spx_server>();
    spx_status st = served_data(ctx, points, indexes, n_indexes, srv->data);
    if (st != SPX_OK)
        return st;
    if (reinterpret_cast<uintptr_t>(srv->data.pts) & 15)
        return ctx_error(ctx, SPX_EINVAL, "server: point buffer must be 16-byte aligned");
    cudaSetDevice(srv->data.device);
    if (!prm.output_budget) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess)
            return ctx_error(ctx, SPX_ECUDA, "server: cudaMemGetInfo failed");
        prm.output_budget = fr / 2;
    }
    srv->prm = prm;
    srv->max_batch = prm.max_batch;
    srv->t0 = Clock::now();
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = srv->data.device;
    if (cudaMemPoolCreate(&srv->pool, &pp) != cudaSuccess)
        return ctx_error(ctx, SPX_ECUDA, "server: cudaMemPoolCreate failed");
    uint64_t keep = UINT64_MAX; // keep freed blocks in the pool
    cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    auto cleanup = [&](const char *what) {
        for (auto &sl : srv->slots) {
            if (sl->s)
                cudaStreamDestroy(sl->s);
            cudaFree(sl->scratch);
            cudaFree(sl->dev_words);
            cudaFreeHost(sl->host_words);
        }
        if (srv->release_stream)
            cudaStreamDestroy(srv->release_stream);
        cudaMemPoolDestroy(srv->pool);
        return ctx_error(ctx, SPX_ENOMEM, std::string("server: ") + what);
    };
    if (cudaStreamCreateWithFlags(&srv->release_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup("stream creation failed");
    // per-request passes take their join scratch from the pool per batch
    const size_t scratch = prm.plain   ? plain_split_scratch_bytes(srv->data.n)
                           : prm.fused ? multi_scratch_bytes(srv->data.n, kMaxBatch)
                                       : 16;
    for (int i = 0; i < prm.slots; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->srv = srv.get();
        Slot *p = sl.get();
        srv->slots.push_back(std::move(sl));
        if (cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking) != cudaSuccess)
            return cleanup("stream creation failed");
        if (cudaMalloc(&p->scratch, scratch) != cudaSuccess)
            return cleanup("scratch allocation failed");
        const size_t words = kWordStats + kStatCount;
        if (cudaMalloc(reinterpret_cast<void **>(&p->dev_words), words * 8) != cudaSuccess ||
            cudaMemset(p->dev_words, 0, words * 8) != cudaSuccess)
            return cleanup("status words allocation failed");
        if (cudaMallocHost(reinterpret_cast<void **>(&p->host_words), (kMaxBatch + 1) * 8) != cudaSuccess)
            return cleanup("pinned allocation failed");
    }
    spx_server *raw = srv.get();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = srv.release();
    return SPX_OK;
}

spx_status spx_server_submit(spx_server *srv, const spx_request *req, uint64_t *req_id)
{
    if (!srv || !req || !req_id)
        return SPX_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (req->kind != SPX_REQ_SELECT && req->kind != SPX_REQ_JOIN) {
        srv->err = "server: request kind must be SPX_REQ_SELECT or SPX_REQ_JOIN";
        return SPX_EINVAL;
    }
    if (req->index >= srv->data.ix.size()) {
        srv->err = "server: request index position out of range";
        return SPX_EINVAL;
    }
    const uint32_t P = srv->data.ix[req->index].P;
    if (req->kind == SPX_REQ_SELECT && P > kSelectMaxQueries) {
        srv->err = "server: a selection index has at most 1024 polygons";
        return SPX_EINVAL;
    }
    if (srv->stopping) {
        srv->err = "server: stopping";
        return SPX_EINVAL;
    }
    auto r = std::make_unique<Req>();
    r->id = srv->next_id++;
    r->rq = *req;
    r->P = P;
    r->t_submit = srv->now_ms();
    srv->queue.push_back(r.get());
    *req_id = r->id;
    srv->reqs[r->id] = std::move(r);
    srv->st.submitted++;
    srv->signal();
    return SPX_OK;
}

spx_status spx_server_submit_polygons(spx_server *srv, int kind, const int32_t *xy, const uint64_t *ring_off,
                                      uint32_t P, uint64_t tag, uint64_t *req_id)
{
    if (!srv || !req_id || !ring_off || (P && !xy))
        return SPX_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (kind != SPX_REQ_SELECT && kind != SPX_REQ_JOIN) {
        srv->err = "server: request kind must be SPX_REQ_SELECT or SPX_REQ_JOIN";
        return SPX_EINVAL;
    }
    if (kind == SPX_REQ_SELECT && P > kSelectMaxQueries) {
        srv->err = "server: a selection has at most 1024 polygons";
        return SPX_EINVAL;
    }
    const std::string bad = check_rings(xy, ring_off, P);
    if (!bad.empty()) {
        srv->err = "server: " + bad;
        return SPX_EINVAL;
    }
    if (srv->stopping) {
        srv->err = "server: stopping";
        return SPX_EINVAL;
    }
    auto r = std::make_unique<Req>();
    r->id = srv->next_id++;
    r->rq.kind = kind;
    r->rq.tag = tag;
    r->P = P;
    r->own = true;
    r->off.assign(ring_off, ring_off + P + 1);
    r->xy.assign(xy, xy + 2 * (P ? ring_off[P] : 0));
    r->t_submit = srv->now_ms();
    srv->queue.push_back(r.get());
    *req_id = r->id;
    srv->reqs[r->id] = std::move(r);
    srv->st.submitted++;
    srv->signal();
    return SPX_OK;
}

static void fill_result(const Req &r, spx_result *out)
{
    std::memset(out, 0, sizeof(*out));
    out->status = r.status;
    out->kind = r.rq.kind;
    out->tag = r.rq.tag;
    out->total = r.total;
    out->n_polys = r.P;
    out->batch_size = r.batch_size;
    if (r.status == SPX_OK) {
        if (r.rq.kind == SPX_REQ_JOIN) {
            out->pairs_dev = static_cast<const uint32_t *>(r.out_mem);
            out->counts_dev = reinterpret_cast<const uint64_t *>(r.counts);
        } else {
            const char *o = static_cast<const char *>(r.out_mem);
            out->ids_dev = reinterpret_cast<const uint32_t *>(o);
            out->offsets_dev = reinterpret_cast<const uint64_t *>(o + up256(std::max<uint64_t>(r.total, 1) * 4));
        }
    }
    out->t_submit_ms = r.t_submit;
    out->t_start_ms = r.t_start;
    out->t_done_ms = r.t_done;
    out->t_counted_ms = r.t_counted;
    out->t_written_ms = r.t_written;
}

spx_status spx_server_poll(spx_server *srv, uint64_t req_id, spx_result *out)
{
    return spx_server_wait(srv, req_id, 0.0, out);
}

spx_status spx_server_wait(spx_server *srv, uint64_t req_id, double timeout_ms, spx_result *out)
{
    if (!srv || !out)
        return SPX_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) {
        srv->err = "server: unknown request id";
        return SPX_EINVAL;
    }
    Req *r = it->second.get();
    auto ready = [&] { return r->status != SPX_EBUSY; };
    if (timeout_ms < 0)
        srv->cv_done.wait(lk, ready);
    else if (timeout_ms > 0)
        srv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
    if (!ready())
        return SPX_EBUSY;
    fill_result(*r, out);
    return SPX_OK;
}

spx_status spx_server_read(spx_server *srv, uint64_t req_id, void *a, uint64_t a_bytes, void *b, uint64_t b_bytes)
{
    if (!srv)
        return SPX_EINVAL;
    spx_result r{};
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(req_id);
        if (it == srv->reqs.end()) {
            srv->err = "server: unknown request id";
            return SPX_EINVAL;
        }
        if (it->second->status == SPX_EBUSY)
            return SPX_EBUSY;
        if (it->second->status != SPX_OK) {
            srv->err = "server: the request failed; there is no result to read";
            return SPX_EINVAL;
        }
        fill_result(*it->second, &r);
        it->second->readers++; // keeps release from freeing the outputs during the copy
    }
    auto done_reading = [&]() {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto jt = srv->reqs.find(req_id);
        if (jt != srv->reqs.end())
            jt->second->readers--;
    };
    const bool join = r.kind == SPX_REQ_JOIN;
    const uint64_t na = join ? r.total * 8 : r.total * 4;
    const uint64_t nb = join ? uint64_t(r.n_polys) * 8 : (uint64_t(r.n_polys) + 1) * 8;
    if ((a && a_bytes < na) || (b && b_bytes < nb)) {
        done_reading();
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->err = "server: read buffer too small";
        return SPX_ECAPACITY;
    }
    // outside the mutex: a blocking copy (stream callbacks take the mutex)
    cudaSetDevice(srv->data.device);
    const void *src_a = join ? static_cast<const void *>(r.pairs_dev) : static_cast<const void *>(r.ids_dev);
    const void *src_b = join ? static_cast<const void *>(r.counts_dev) : static_cast<const void *>(r.offsets_dev);
    cudaError_t e = cudaSuccess;
    if (a && na)
        e = cudaMemcpy(a, src_a, na, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && b && nb)
        e = cudaMemcpy(b, src_b, nb, cudaMemcpyDeviceToHost);
    done_reading();
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->err = std::string("server: read copy failed: ") + cudaGetErrorString(e);
        return SPX_ECUDA;
    }
    return SPX_OK;
}

spx_status spx_server_release(spx_server *srv, uint64_t req_id)
{
    if (!srv)
        return SPX_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) {
        srv->err = "server: unknown request id";
        return SPX_EINVAL;
    }
    Req *r = it->second.get();
    if (r->status == SPX_EBUSY)
        return SPX_EBUSY;
    if (r->readers > 0) {
        srv->err = "server: a read of this request is in progress; release it after the read returns";
        return SPX_EBUSY;
    }
    pool_free(r->out_mem, srv->release_stream);
    pool_free(r->counts, srv->release_stream);
    srv->used -= r->out_bytes + r->counts_bytes;
    srv->reqs.erase(it);
    srv->signal(); // a batch may be waiting for budget
    return SPX_OK;
}

spx_status spx_server_stats(spx_server *srv, spx_server_stats_t *out)
{
    if (!srv || !out)
        return SPX_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    out->bytes_in_use = srv->used;
    return SPX_OK;
}

const char *spx_server_last_error(spx_server *srv)
{
    static thread_local std::string copy;
    if (!srv)
        return "null server";
    std::lock_guard<std::mutex> lk(srv->mu);
    copy = srv->err;
    return copy.c_str();
}

void spx_server_destroy(spx_server *srv)
{
    if (!srv)
        return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->signal();
    if (srv->worker.joinable())
        srv->worker.join();
    cudaSetDevice(srv->data.device);
    for (auto &kv : srv->reqs) {
        Req *r = kv.second.get();
        pool_free(r->out_mem, srv->release_stream);
        pool_free(r->tmp_mem, srv->release_stream);
        pool_free(r->counts, srv->release_stream);
        pool_free(r->own_mem, srv->release_stream);
    }
    cudaStreamSynchronize(srv->release_stream);
    for (auto &sl : srv->slots) {
        cudaStreamSynchronize(sl->s);
        cudaStreamDestroy(sl->s);
        cudaFree(sl->scratch);
        cudaFree(sl->dev_words);
        cudaFreeHost(sl->host_words);
    }
    cudaStreamDestroy(srv->release_stream);
    cudaMemPoolDestroy(srv->pool);
    delete srv;
}

} // extern "C"
