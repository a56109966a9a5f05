// gc_server.cu -- request loop over several resident graphs (include/gc.h,
// "Serving").  Host code only: every batch runs through gc_apply_batch on its
// graph's own stream, so batches of different graphs overlap on the device.
//
// Scheduling: per-graph FIFO queues; `slots` worker threads.  A free worker
// takes the oldest queued request whose graph is idle and whose predicted
// device-memory growth fits the budget (after releasing the scratch of idle
// graphs if needed).  Requests of one graph never overlap, which keeps the
// per-graph order of Algorithm 2's commits.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "gc.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    gc_result r{};
    std::vector<int32_t> ins, del;
    bool done = false;
};

}  // namespace

struct gc_server {
    std::vector<gc_graph*> graphs;
    std::vector<std::deque<Request*>> queue;
    std::vector<char> busy;
    std::vector<long long> held;  // gc_device_bytes of each graph when idle
    long long budget = 0;
    long long inflight_pred = 0;
    int running = 0;
    long long peak_running = 0;
    long long trims = 0;
    long long pending = 0;        // submitted and not yet done
    std::unordered_map<long long, Request*> reqs;
    long long next_ticket = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    Clock::time_point t0;
};

namespace {

double ms_since(const gc_server* s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

long long held_total(const gc_server* s) {
    long long t = 0;
    for (long long h : s->held) t += h;
    return t;
}

// Choose the next request under the lock; nullptr if none can start now.
Request* pick(gc_server* s, int* gi) {
    for (;;) {
        // oldest head among idle graphs
        int best = -1;
        for (int i = 0; i < (int)s->graphs.size(); i++) {
            if (s->busy[i] || s->queue[i].empty()) continue;
            if (best < 0 || s->queue[i].front()->r.ticket < s->queue[best].front()->r.ticket) best = i;
        }
        if (best < 0) return nullptr;
        Request* q = s->queue[best].front();
        const long long pred = gc_batch_bytes(s->graphs[best], q->r.n_ins, q->r.n_del);
        q->r.bytes_predicted = pred;
        if (held_total(s) + s->inflight_pred + pred <= s->budget || s->running == 0) {
            // a request that cannot fit even alone still runs when nothing else does
            if (held_total(s) + s->inflight_pred + pred > s->budget) {
                // release what idle graphs hold before running it alone
                for (int i = 0; i < (int)s->graphs.size(); i++) {
                    if (i == best || s->busy[i]) continue;
                    long long before = s->held[i];
                    gc_trim(s->graphs[i]);
                    s->held[i] = gc_device_bytes(s->graphs[i]);
                    if (s->held[i] < before) s->trims++;
                }
            }
            *gi = best;
            return q;
        }
        // does not fit: release the scratch of idle graphs, largest first
        std::vector<int> idle;
        for (int i = 0; i < (int)s->graphs.size(); i++)
            if (i != best && !s->busy[i]) idle.push_back(i);
        std::sort(idle.begin(), idle.end(), [&](int a, int b) { return s->held[a] > s->held[b]; });
        bool freed = false;
        for (int i : idle) {
            long long before = s->held[i];
            gc_trim(s->graphs[i]);
            s->held[i] = gc_device_bytes(s->graphs[i]);
            if (s->held[i] < before) {
                s->trims++;
                freed = true;
                if (held_total(s) + s->inflight_pred + pred <= s->budget) break;
            }
        }
        if (!freed || held_total(s) + s->inflight_pred + pred > s->budget) return nullptr;  // wait for running ones
    }
}

void worker(gc_server* s) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        int gi = -1;
        Request* q = pick(s, &gi);
        if (!q) {
            if (s->stop && s->pending == 0) return;
            s->cv_work.wait(lk);
            continue;
        }
        s->queue[gi].pop_front();
        s->busy[gi] = 1;
        s->inflight_pred += q->r.bytes_predicted;
        s->running++;
        s->peak_running = std::max<long long>(s->peak_running, s->running);
        q->r.t_admit_ms = ms_since(s);
        gc_graph* g = s->graphs[gi];
        lk.unlock();

        const int32_t* ins = q->ins.empty() ? nullptr : q->ins.data();
        const int32_t* del = q->del.empty() ? nullptr : q->del.data();
        const long long n_ins = q->r.n_ins, n_del = q->r.n_del;
        q->r.status = gc_apply_batch(g, ins, n_ins, del, n_del, q->r.counts);
        gc_stats st{};
        if (gc_batch_stats(g, &st) == GC_OK && q->r.status == GC_OK) {
            q->r.n_ins = st.n_ins;
            q->r.n_del = st.n_del;
            q->r.region_vertices = st.region_vertices;
            q->r.ms_device = st.ms_device;
            q->r.relayouts = st.relayouts;
        }
        const long long h = gc_device_bytes(g);
        std::vector<int32_t>().swap(q->ins);
        std::vector<int32_t>().swap(q->del);

        lk.lock();
        s->busy[gi] = 0;
        s->held[gi] = h;
        s->inflight_pred -= q->r.bytes_predicted;
        s->running--;
        s->pending--;
        q->r.t_done_ms = ms_since(s);
        q->done = true;
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

int gc_server_open(gc_graph* const* graphs, int32_t n_graphs, const gc_server_options* opt, gc_server** out) {
    if (!out || n_graphs <= 0 || !graphs) return GC_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n_graphs; i++)
        if (!graphs[i]) return GC_EINVAL;
    gc_server_options o{};
    if (opt) o = *opt;
    if (o.slots <= 0) o.slots = 4;
    if (o.slots > 64) return GC_EINVAL;
    gc_server* s = new gc_server();
    s->t0 = Clock::now();
    s->graphs.assign(graphs, graphs + n_graphs);
    s->queue.resize(n_graphs);
    s->busy.assign(n_graphs, 0);
    s->held.resize(n_graphs);
    for (int i = 0; i < n_graphs; i++) s->held[i] = gc_device_bytes(graphs[i]);
    if (o.hbm_budget_bytes > 0) {
        s->budget = o.hbm_budget_bytes;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return GC_ECUDA;
        }
        s->budget = held_total(s) + (long long)(0.9 * (double)fr);
    }
    for (int i = 0; i < o.slots; i++) s->workers.emplace_back(worker, s);
    *out = s;
    return GC_OK;
}

int gc_server_submit(gc_server* s, int32_t graph, const int32_t* ins, int64_t n_ins, const int32_t* del,
                     int64_t n_del, int64_t* ticket) {
    if (!s || !ticket || graph < 0 || graph >= (int32_t)s->graphs.size() || n_ins < 0 || n_del < 0 ||
        (n_ins > 0 && !ins) || (n_del > 0 && !del))
        return GC_EINVAL;
    Request* q = new Request();
    q->ins.assign(ins, ins + 2 * n_ins);
    q->del.assign(del, del + 2 * n_del);
    q->r.graph = graph;
    q->r.n_ins = n_ins;
    q->r.n_del = n_del;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete q;
        return GC_EINVAL;
    }
    q->r.ticket = s->next_ticket++;
    q->r.t_submit_ms = ms_since(s);
    s->reqs[q->r.ticket] = q;
    s->queue[graph].push_back(q);
    s->pending++;
    *ticket = q->r.ticket;
    s->cv_work.notify_one();
    return GC_OK;
}

int gc_server_wait(gc_server* s, int64_t ticket, gc_result* r) {
    if (!s) return GC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return GC_EINVAL;
    Request* q = it->second;
    s->cv_done.wait(lk, [&] { return q->done; });
    if (r) *r = q->r;
    s->reqs.erase(ticket);
    delete q;
    return GC_OK;
}

int gc_server_drain(gc_server* s) {
    if (!s) return GC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending == 0; });
    return GC_OK;
}

int gc_server_counters(const gc_server* s, int64_t* peak_inflight, int64_t* trims) {
    if (!s) return GC_EINVAL;
    gc_server* m = const_cast<gc_server*>(s);
    std::lock_guard<std::mutex> lk(m->mu);
    if (peak_inflight) *peak_inflight = s->peak_running;
    if (trims) *trims = s->trims;
    return GC_OK;
}

void gc_server_close(gc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
