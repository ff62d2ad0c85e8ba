// Serving loop: requests (raw edge pairs + eps) arrive at any time and are
// answered by continuous batching on one GPU.
//
//   submit  copies the request into host memory the server owns and queues
//           it (DSG_EBUSY when the queue is full: back-pressure);
//   worker  (one host thread per server) admits queued requests while their
//           device-memory charge fits the budget and hands them to the
//           ingest threads, and whenever one of its max_inflight solve
//           streams is free launches one block-per-graph launch over
//           everything ingested so far on that stream; while batches run,
//           new arrivals keep being admitted and ingested, and form the next
//           batch; a finished batch's results are copied out, its graphs
//           freed and their charge returned to the budget;
//   ingest  (ingest_threads host threads, each with its own stream) turn
//           admitted requests into resident graphs; a request above
//           big_work goes to the big-request thread, the rest to the batches;
//   big     (big_threads host threads, each with its own stream) solve big
//           requests one at a time each with the grid-wide kernels on big_sms
//           SMs (the batches get the others), so one large graph never holds
//           a batch of small ones back;
//   poll    waits (bounded) for one ticket's completion.
// A request's results do not depend on what it is batched with: each graph is
// solved by its own block with its own state.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dsg_batch.cuh"
#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

static double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeReq {
    uint64_t ticket = 0;
    uint32_t n = 0;
    uint64_t m_raw = 0;
    uint32_t* src = nullptr;  // host copy (freed after ingest) or the caller's borrowed arrays
    uint32_t* dst = nullptr;
    bool owned = true;
    uint32_t p = 0, q = 1;
    bool want_core = false;
    uint8_t* out_set = nullptr;  // caller's host buffers
    uint32_t* core = nullptr;
    double t_submit = 0, t_done = 0;
    bool done = false;
    dsg_status status = DSG_OK;
    uint64_t res[4] = {0, 0, 0, 0};
    uint64_t m = 0;
    dsg_graph* g = nullptr;
    size_t charge = 0;
};

}  // namespace dsg

struct dsg_server {
    dsg_serve_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<dsg::ServeReq*> pending;
    std::vector<dsg::ServeReq*> ready;
    std::unordered_map<uint64_t, dsg::ServeReq*> by_ticket;
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    bool stop = false;
    std::thread worker;
    std::vector<cudaStream_t> s_solve;  // one per batch that may be in flight
    // ingest threads and the big-request thread
    std::condition_variable cv_ingest, cv_big;
    std::deque<dsg::ServeReq*> to_ingest, big;
    std::vector<std::thread> ingesters;
    std::vector<cudaStream_t> s_ingest;
    std::vector<std::thread> big_workers;
    std::vector<cudaStream_t> s_big;
    bool stop_helpers = false;
    // statistics
    uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, batches = 0, big_done = 0;
    double ingest_busy_us = 0, big_busy_us = 0, batch_dev_ms = 0;
    std::vector<double> lat_us;
    double t0 = 0;
};

namespace dsg {

// device bytes a request may hold while resident: raw pairs during ingest
// (8 per pair), ingest temporaries (two bucket passes of 16 per pair, the
// unsorted rows 8 per pair, per-vertex arrays), the CSR and the batch scratch
static size_t request_charge(uint32_t n, uint64_t m_raw) {
    return (size_t)m_raw * 64 + (size_t)n * 96 + (64u << 10);
}

struct Inflight {
    std::vector<ServeReq*> reqs;
    BatchArgs a;
    uint64_t* d_res = nullptr;
    uint32_t* d_tables = nullptr;  // one allocation for every table and scratch array
    size_t tables_bytes = 0;
    std::vector<uint64_t> slot;
    uint64_t N = 0;
    cudaEvent_t start_ev = nullptr, done_ev = nullptr;
};

static void finish_request(dsg_server* s, ServeReq* r, dsg_status st) {
    r->status = st;
    r->t_done = now_us();
    if (r->g) {
        dsg_graph_free(r->g);
        r->g = nullptr;
    }
    if (r->owned) {
        free(r->src);
        free(r->dst);
    }
    r->src = r->dst = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= r->charge;
    r->done = true;
    s->completed++;
    s->lat_us.push_back(r->t_done - r->t_submit);
    s->cv_done.notify_all();
}

static bool is_big(const dsg_server* s, const ServeReq* r) {
    return s->cfg.big_work != UINT64_MAX && 2 * r->m_raw + r->n > s->cfg.big_work;
}

// Ingest one admitted request on stream st (synchronous for that stream only)
// and hand it to the batches or to the big-request thread.
static void ingest_one(dsg_server* s, ServeReq* r, cudaStream_t st_ing) {
    const double t_in = now_us();
    dsg_graph* g = nullptr;
    dsg_status st = dsg_graph_from_edges(r->n, r->m_raw, r->src, r->dst, 0, st_ing, &g);
    if (r->owned) {
        free(r->src);
        free(r->dst);
    }
    r->src = r->dst = nullptr;
    if (st != DSG_OK) {
        finish_request(s, r, st);
        return;
    }
    r->g = g;
    r->m = g->m;
    const bool big = is_big(s, r);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->ingest_busy_us += now_us() - t_in;
        if (big) s->big.push_back(r);
        else s->ready.push_back(r);
    }
    if (big) s->cv_big.notify_one();
    else s->cv_work.notify_one();
}

static void ingest_main(dsg_server* s, cudaStream_t st) {
    cudaSetDevice(s->device);
    for (;;) {
        ServeReq* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_ingest.wait(lk, [&] { return s->stop_helpers || !s->to_ingest.empty(); });
            if (s->to_ingest.empty()) return;  // stopping, nothing left
            r = s->to_ingest.front();
            s->to_ingest.pop_front();
        }
        ingest_one(s, r, st);
    }
}

// A big request alone: the peel (and core numbers) by the grid-wide kernels,
// capped at big_sms blocks of one per SM, on the big stream.
static void solve_big(dsg_server* s, ServeReq* r, cudaStream_t sb) {
    const double t_in = now_us();
    dsg_graph view = *r->g;
    view.owns = false;
    view.stream = sb;
    view.max_blocks = s->cfg.big_sms;
    view.force_block = 1024;
    dsg_status st = DSG_OK;
    uint8_t* set_dev = nullptr;
    if (r->out_set && r->n) {
        if (dev_alloc((void**)&set_dev, r->n, sb) != cudaSuccess) st = DSG_ENOMEM;
    }
    if (st == DSG_OK) st = peel_into(&view, r->p, r->q, set_dev, r->res);
    if (st == DSG_OK && r->out_set && r->n &&
        (cudaMemcpyAsync(r->out_set, set_dev, r->n, cudaMemcpyDeviceToHost, sb) != cudaSuccess ||
         cudaStreamSynchronize(sb) != cudaSuccess))
        st = DSG_ECUDA;
    if (set_dev) dev_free(set_dev, sb);
    if (st == DSG_OK && r->want_core && r->core && r->n) st = run_kcore(&view, r->core, nullptr, 0);
    cudaStreamSynchronize(sb);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->big_busy_us += now_us() - t_in;
        s->big_done++;
    }
    finish_request(s, r, st);
}

static void big_main(dsg_server* s, cudaStream_t sb) {
    cudaSetDevice(s->device);
    for (;;) {
        ServeReq* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_big.wait(lk, [&] { return s->stop_helpers || !s->big.empty(); });
            if (s->big.empty()) return;
            r = s->big.front();
            s->big.pop_front();
        }
        solve_big(s, r, sb);
        s->cv_work.notify_one();
    }
}

// Build the tables of one batch and launch it on the solve stream.
static dsg_status launch_batch(dsg_server* s, Inflight& f, cudaStream_t ss) {
    const uint32_t G = (uint32_t)f.reqs.size();
    // largest first inside the batch
    std::stable_sort(f.reqs.begin(), f.reqs.end(), [](ServeReq* x, ServeReq* y) {
        return 2 * x->m + x->n > 2 * y->m + y->n;
    });
    f.slot.resize(G + 1);
    f.slot[0] = 0;
    for (uint32_t i = 0; i < G; ++i) f.slot[i + 1] = f.slot[i] + f.reqs[i]->n;
    f.N = f.slot[G];
    const uint64_t N = f.N ? f.N : 1;
    // one allocation: tables + scratch + outputs
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_goff = carve(G * sizeof(void*)), o_gadj = carve(G * sizeof(void*)), o_slot = carve(G * 8),
                 o_gn = carve(G * 4), o_p = carve(G * 4), o_q = carve(G * 4), o_wc = carve(G), o_order = carve(G * 4),
                 o_st = carve(N * 4), o_la = carve(N * 4), o_lb = carve(N * 4), o_lf = carve(N * 4),
                 o_core = carve(N * 4), o_set = carve(N), o_res = carve(4 * (size_t)G * 8), o_next = carve(8);
    f.tables_bytes = off;
    DSG_TRY_CUDA(dev_alloc((void**)&f.d_tables, off, ss));
    unsigned char* base = reinterpret_cast<unsigned char*>(f.d_tables);
    std::vector<unsigned char> host(o_st, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) { memcpy(host.data() + o, src, bytes); };
    std::vector<const uint64_t*> goff(G);
    std::vector<const uint32_t*> gadj(G);
    std::vector<uint32_t> gn(G), gp(G), gq(G), order(G);
    std::vector<uint8_t> wc(G);
    for (uint32_t i = 0; i < G; ++i) {
        ServeReq* r = f.reqs[i];
        goff[i] = r->g->off;
        gadj[i] = r->g->adj;
        gn[i] = r->n;
        gp[i] = r->p;
        gq[i] = r->q;
        wc[i] = r->want_core ? 1 : 0;
        order[i] = i;
    }
    put(o_goff, goff.data(), G * sizeof(void*));
    put(o_gadj, gadj.data(), G * sizeof(void*));
    put(o_slot, f.slot.data(), G * 8);
    put(o_gn, gn.data(), G * 4);
    put(o_p, gp.data(), G * 4);
    put(o_q, gq.data(), G * 4);
    put(o_wc, wc.data(), G);
    put(o_order, order.data(), G * 4);
    DSG_TRY_CUDA(cudaMemcpyAsync(base, host.data(), o_st, cudaMemcpyHostToDevice, ss));
    DSG_TRY_CUDA(cudaMemsetAsync(base + o_next, 0, 8, ss));
    DSG_TRY_CUDA(cudaEventCreate(&f.start_ev));
    DSG_TRY_CUDA(cudaEventRecord(f.start_ev, ss));
    BatchArgs& a = f.a;
    a.G = G;
    a.goff = reinterpret_cast<const uint64_t* const*>(base + o_goff);
    a.gadj = reinterpret_cast<const uint32_t* const*>(base + o_gadj);
    a.slot = reinterpret_cast<const uint64_t*>(base + o_slot);
    a.gn = reinterpret_cast<const uint32_t*>(base + o_gn);
    a.p = reinterpret_cast<const uint32_t*>(base + o_p);
    a.q = reinterpret_cast<const uint32_t*>(base + o_q);
    a.want_core = reinterpret_cast<const uint8_t*>(base + o_wc);
    a.order = reinterpret_cast<const uint32_t*>(base + o_order);
    a.st = reinterpret_cast<uint32_t*>(base + o_st);
    a.la = reinterpret_cast<uint32_t*>(base + o_la);
    a.lb = reinterpret_cast<uint32_t*>(base + o_lb);
    a.lf = reinterpret_cast<uint32_t*>(base + o_lf);
    a.core = reinterpret_cast<uint32_t*>(base + o_core);
    a.out_set = reinterpret_cast<uint8_t*>(base + o_set);
    a.res = reinterpret_cast<uint64_t*>(base + o_res);
    a.next = reinterpret_cast<unsigned long long*>(base + o_next);
    a.hot_deg = 0;
    a.stats = nullptr;
    f.d_res = a.res;
    // the batches leave the big-request threads' share of the SMs free
    const uint32_t sms = (uint32_t)dev_info().sms;
    const uint32_t big_sms =
        s->cfg.big_work == UINT64_MAX ? 0 : (uint32_t)std::min<uint64_t>((uint64_t)s->cfg.big_sms * s->cfg.big_threads, sms - 1);
    const uint32_t cap = (uint32_t)((uint64_t)batch_slots_for(512) * (sms - big_sms) / sms);
    DSG_TRY_CUDA(batch_launch(a, ss, 512, cap ? cap : 1));
    DSG_TRY_CUDA(cudaEventCreate(&f.done_ev));
    DSG_TRY_CUDA(cudaEventRecord(f.done_ev, ss));
    // (the pageable staging vector may go: a host-to-device copy from pageable
    // memory has consumed its source when cudaMemcpyAsync returns)
    return DSG_OK;
}

// Copy a finished batch's results out and release its requests.
static void complete_batch(dsg_server* s, Inflight& f, cudaStream_t ss) {
    const uint32_t G = (uint32_t)f.reqs.size();
    std::vector<uint64_t> res(4 * (size_t)G);
    dsg_status st = DSG_OK;
    if (cudaMemcpyAsync(res.data(), f.d_res, res.size() * 8, cudaMemcpyDeviceToHost, ss) != cudaSuccess)
        st = DSG_ECUDA;
    for (uint32_t i = 0; i < G && st == DSG_OK; ++i) {
        ServeReq* r = f.reqs[i];
        if (r->out_set && r->n &&
            cudaMemcpyAsync(r->out_set, f.a.out_set + f.slot[i], r->n, cudaMemcpyDeviceToHost, ss) != cudaSuccess)
            st = DSG_ECUDA;
        if (r->core && r->want_core && r->n &&
            cudaMemcpyAsync(r->core, f.a.core + f.slot[i], (size_t)r->n * 4, cudaMemcpyDeviceToHost, ss) !=
                cudaSuccess)
            st = DSG_ECUDA;
    }
    if (cudaStreamSynchronize(ss) != cudaSuccess) st = DSG_ECUDA;
    for (uint32_t i = 0; i < G; ++i) {
        ServeReq* r = f.reqs[i];
        for (int k = 0; k < 4; ++k) r->res[k] = res[4 * (size_t)i + k];
        finish_request(s, r, st);
    }
    float dev_ms = 0;
    if (cudaEventElapsedTime(&dev_ms, f.start_ev, f.done_ev) != cudaSuccess) dev_ms = 0;
    dev_free(f.d_tables, ss);
    cudaEventDestroy(f.start_ev);
    cudaEventDestroy(f.done_ev);
    f = Inflight();
    std::lock_guard<std::mutex> lk(s->mu);
    s->batches++;
    s->batch_dev_ms += dev_ms;
}

static void worker_main(dsg_server* s) {
    cudaSetDevice(s->device);
    const size_t K = s->s_solve.size();
    std::vector<Inflight> fl(K);
    std::vector<bool> running(K, false);
    auto any_running = [&]() {
        for (size_t k = 0; k < K; ++k)
            if (running[k]) return true;
        return false;
    };
    for (;;) {
        size_t admitted_now = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (!any_running() && s->pending.empty() && s->ready.empty()) {
                // stop once every admitted request has completed (ingest and big threads included)
                if (s->stop && s->admitted == s->completed) break;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            // admit in arrival order while the budget allows; the ingest threads take them
            while (!s->pending.empty()) {
                ServeReq* r = s->pending.front();
                if (s->in_use + r->charge > s->cfg.hbm_budget && s->in_use > 0) break;
                s->pending.pop_front();
                s->in_use += r->charge;
                s->admitted++;
                s->to_ingest.push_back(r);
                ++admitted_now;
            }
        }
        if (admitted_now) s->cv_ingest.notify_all();
        // finished batches: results out, memory back
        for (size_t k = 0; k < K; ++k) {
            if (running[k] && cudaEventQuery(fl[k].done_ev) != cudaErrorNotReady) {
                complete_batch(s, fl[k], s->s_solve[k]);
                running[k] = false;
            }
        }
        // continuous batching: whatever is ready goes to a free batch slot now
        for (size_t k = 0; k < K; ++k) {
            if (running[k]) continue;
            std::vector<ServeReq*> batch;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                // in arrival order, at most max_batch graphs and max_batch_work of work (at least one)
                size_t take = 0;
                uint64_t work = 0;
                while (take < s->ready.size() && take < s->cfg.max_batch) {
                    const ServeReq* r = s->ready[take];
                    const uint64_t w = 2 * r->m + r->n;
                    if (take > 0 && work + w > s->cfg.max_batch_work) break;
                    work += w;
                    ++take;
                }
                batch.assign(s->ready.begin(), s->ready.begin() + take);
                s->ready.erase(s->ready.begin(), s->ready.begin() + take);
            }
            if (batch.empty()) break;
            fl[k].reqs = batch;
            dsg_status st = launch_batch(s, fl[k], s->s_solve[k]);
            if (st != DSG_OK) {
                for (ServeReq* r : fl[k].reqs) finish_request(s, r, st);
                if (fl[k].d_tables) dev_free(fl[k].d_tables, s->s_solve[k]);
                if (fl[k].start_ev) cudaEventDestroy(fl[k].start_ev);
                if (fl[k].done_ev) cudaEventDestroy(fl[k].done_ev);
                fl[k] = Inflight();
            } else {
                running[k] = true;
            }
        }
        {
            // wait a little for arrivals, ingests or completions rather than spin
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->pending.empty() && s->ready.empty()) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
        }
    }
    for (size_t k = 0; k < K; ++k)
        if (running[k]) complete_batch(s, fl[k], s->s_solve[k]);
}

}  // namespace dsg

using namespace dsg;

extern "C" {

dsg_status dsg_serve_create(const dsg_serve_config* cfg, dsg_server** out) {
    clear_error();
    DSG_CHECK_ARG(out, "out is NULL");
    dsg_server* s = new dsg_server();
    if (cfg) s->cfg = *cfg;
    else memset(&s->cfg, 0, sizeof(s->cfg));
    if (!s->cfg.max_batch) s->cfg.max_batch = 1024;
    if (!s->cfg.max_batch_work) s->cfg.max_batch_work = UINT64_MAX;
    if (!s->cfg.max_pending) s->cfg.max_pending = 1u << 16;
    if (!s->cfg.max_inflight) s->cfg.max_inflight = 4;
    if (!s->cfg.ingest_threads) s->cfg.ingest_threads = 4;
    if (!s->cfg.big_work) s->cfg.big_work = 1ull << 23;
    if (!s->cfg.big_threads) s->cfg.big_threads = 2;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess && !s->cfg.hbm_budget) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        s->cfg.hbm_budget = fr / 2;
    }
    if (e == cudaSuccess && !s->cfg.big_sms)
        s->cfg.big_sms = std::max<uint32_t>(1, (uint32_t)dev_info().sms / (4 * s->cfg.big_threads));
    s->s_ingest.assign(s->cfg.ingest_threads, nullptr);
    for (uint32_t k = 0; k < s->cfg.ingest_threads && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithFlags(&s->s_ingest[k], cudaStreamNonBlocking);
    s->s_big.assign(s->cfg.big_threads, nullptr);
    for (uint32_t k = 0; k < s->cfg.big_threads && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithFlags(&s->s_big[k], cudaStreamNonBlocking);
    s->s_solve.assign(s->cfg.max_inflight, nullptr);
    for (uint32_t k = 0; k < s->cfg.max_inflight && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithFlags(&s->s_solve[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        set_error("serve_create: %s", cudaGetErrorString(e));
        for (cudaStream_t st : s->s_ingest)
            if (st) cudaStreamDestroy(st);
        for (cudaStream_t st : s->s_big)
            if (st) cudaStreamDestroy(st);
        for (cudaStream_t st : s->s_solve)
            if (st) cudaStreamDestroy(st);
        delete s;
        return DSG_ECUDA;
    }
    s->t0 = now_us();
    for (uint32_t k = 0; k < s->cfg.ingest_threads; ++k) s->ingesters.emplace_back(ingest_main, s, s->s_ingest[k]);
    for (uint32_t k = 0; k < s->cfg.big_threads; ++k) s->big_workers.emplace_back(big_main, s, s->s_big[k]);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return DSG_OK;
}

dsg_status dsg_serve_submit(dsg_server* s, const dsg_request* rq, uint64_t* ticket) {
    clear_error();
    DSG_CHECK_ARG(s && rq && ticket, "server / request / ticket is NULL");
    DSG_CHECK_ARG(rq->eps_den != 0, "eps_den must be positive");
    DSG_CHECK_ARG(rq->n < 0x80000000u, "n must be below 2^31");
    DSG_CHECK_ARG(rq->m_raw == 0 || (rq->src && rq->dst), "src/dst is NULL");
    size_t charge = request_charge(rq->n, rq->m_raw);
    DSG_CHECK_ARG(charge <= s->cfg.hbm_budget, "request larger than the server's device-memory budget");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            set_error("serve_submit: server is shutting down");
            return DSG_EBUSY;
        }
        if (s->pending.size() >= s->cfg.max_pending) {
            s->rejected++;
            set_error("serve_submit: queue full (%zu pending)", s->pending.size());
            return DSG_EBUSY;
        }
    }
    ServeReq* r = new ServeReq();
    r->n = rq->n;
    r->m_raw = rq->m_raw;
    r->p = rq->eps_num;
    r->q = rq->eps_den;
    r->want_core = rq->want_core != 0;
    r->out_set = rq->out_set;
    r->core = rq->core;
    r->charge = charge;
    if (rq->flags & DSG_REQ_BORROW) {
        r->owned = false;
        r->src = const_cast<uint32_t*>(rq->src);
        r->dst = const_cast<uint32_t*>(rq->dst);
    } else if (rq->m_raw) {
        r->src = (uint32_t*)malloc(rq->m_raw * 4);
        r->dst = (uint32_t*)malloc(rq->m_raw * 4);
        if (!r->src || !r->dst) {
            free(r->src);
            free(r->dst);
            delete r;
            set_error("serve_submit: host allocation failed");
            return DSG_ENOMEM;
        }
        memcpy(r->src, rq->src, rq->m_raw * 4);
        memcpy(r->dst, rq->dst, rq->m_raw * 4);
    }
    r->t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->by_ticket[r->ticket] = r;
        s->pending.push_back(r);
        s->submitted++;
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return DSG_OK;
}

dsg_status dsg_serve_poll(dsg_server* s, uint64_t ticket, dsg_response* resp, uint32_t timeout_us) {
    clear_error();
    DSG_CHECK_ARG(s && resp, "server / response is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) {
        set_error("serve_poll: unknown ticket %llu", (unsigned long long)ticket);
        return DSG_ENOTFOUND;
    }
    ServeReq* r = it->second;
    if (!r->done && timeout_us)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; });
    if (!r->done) return DSG_EAGAIN;
    resp->status = r->status;
    resp->n = r->n;
    resp->m = r->m;
    resp->E = r->res[0];
    resp->V = r->res[1];
    resp->rounds = r->res[2];
    resp->best_round = r->res[3];
    resp->latency_us = r->t_done - r->t_submit;
    s->by_ticket.erase(it);
    delete r;
    return DSG_OK;
}

dsg_status dsg_serve_stats(dsg_server* s, dsg_serve_info* out) {
    clear_error();
    DSG_CHECK_ARG(s && out, "server / stats is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->pending = s->pending.size();
    out->in_flight = s->admitted - s->completed;
    out->hbm_in_use = s->in_use;
    out->hbm_budget = s->cfg.hbm_budget;
    out->batches = s->batches;
    out->big_done = s->big_done;
    out->ingest_busy_s = s->ingest_busy_us / 1e6;
    out->big_busy_s = s->big_busy_us / 1e6;
    out->batch_device_s = s->batch_dev_ms / 1e3;
    out->uptime_s = (now_us() - s->t0) / 1e6;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->graphs_per_s = out->uptime_s > 0 ? (double)s->completed / out->uptime_s : 0;
    }
    return DSG_OK;
}

void dsg_serve_destroy(dsg_server* s) {
    if (!s) return;
    {
        // requests not yet admitted are cancelled; admitted ones are finished
        std::lock_guard<std::mutex> lk(s->mu);
        s->pending.clear();
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();  // every admitted request completed
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_helpers = true;
    }
    s->cv_ingest.notify_all();
    s->cv_big.notify_all();
    for (auto& t : s->ingesters)
        if (t.joinable()) t.join();
    for (auto& t : s->big_workers)
        if (t.joinable()) t.join();
    for (auto& kv : s->by_ticket) {
        if (kv.second->owned) {
            free(kv.second->src);
            free(kv.second->dst);
        }
        if (kv.second->g) dsg_graph_free(kv.second->g);
        delete kv.second;
    }
    for (cudaStream_t st : s->s_ingest)
        if (st) cudaStreamDestroy(st);
    for (cudaStream_t st : s->s_big)
        if (st) cudaStreamDestroy(st);
    for (cudaStream_t st : s->s_solve)
        if (st) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
