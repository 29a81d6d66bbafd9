// serve.cpp -- qec_stream_*: continuous-batching request loop (include/qec.h).
//
// A stream owns N in-flight slots.  Each slot is one micro-batch: pinned host
// buffers for the windows and results, device copies, its own CUDA stream and
// event, and its own scratch workspace, so micro-batches of different slots run
// concurrently on the device.  One slot at a time is FILLING: qec_stream_submit
// appends the window to it.  A dispatcher thread launches the FILLING slot as
// soon as fewer than N-1 slots are INFLIGHT (immediately when the GPU has room,
// so a lone request is not held back), makes an IDLE slot the new FILLING one,
// and hands out each window's result as soon as the kernel has published it:
// results and per-window completion flags live in pinned host memory mapped
// into the device, so a small window is not held back by the slowest window
// of its micro-batch; a slot is reused once all its windows are out.  A
// micro-batch small enough for one thread block per window is decoded by
// multi-warp teams (a block of TEAM_BIG warps per window), which cuts the
// latency of the large windows; larger micro-batches use one warp per window.

#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "qec_internal.h"

namespace {

int64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

enum { IDLE = 0, FILLING = 1, INFLIGHT = 2 };

struct Slot {
    int state = IDLE;
    int n = 0;
    long long words = 0;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    uint32_t *h_syn = nullptr;
    int32_t *h_gid = nullptr;
    int64_t *h_off = nullptr;
    uint64_t *h_rid = nullptr;
    int64_t *h_tsub = nullptr;
    // results and completion flags: pinned host memory mapped into the device
    // (h_* host addresses, m_* the device's addresses of the same bytes)
    uint64_t *h_obs = nullptr;
    int64_t *h_w = nullptr;
    int32_t *h_st = nullptr;
    int32_t *h_done = nullptr;
    uint64_t *m_obs = nullptr;
    int64_t *m_w = nullptr;
    int32_t *m_st = nullptr;
    int32_t *m_done = nullptr;
    std::vector<int> pending;   // windows of the in-flight micro-batch not yet handed out
    uint32_t *d_syn = nullptr;
    int32_t *d_gid = nullptr;
    int64_t *d_off = nullptr;
    char *slabs = nullptr;
    char *slabs2 = nullptr;
    unsigned long long *queue = nullptr;
    int *overflow = nullptr;
};

int ferr(int code, const std::string &m) { return qec::set_last_error(code, m.c_str()); }

}  // namespace

struct qec_stream {
    int device = 0;
    int nslots = 0;
    int cap_req = 0;
    long long cap_words = 0;
    int max_inflight = 0;
    int nwarps = 0, nwarps2 = 0;
    int team_blocks = 0;   // resident blocks of the TEAM_BIG kernel on the device
    qec::SlabCaps caps{}, caps2{};
    long long sb = 0, sb2 = 0;
    std::vector<Slot> slots;
    std::vector<const qec_graph *> graphs;
    std::vector<qec::DGraph> views;
    std::mutex mu;
    int filling = -1;
    int admitted = 0;
    std::deque<qec_result> done;
    std::atomic<bool> stop{false};
    std::thread th;
    std::string err;
};

namespace {

void free_slot(Slot &s) {
    if (s.cs) cudaStreamSynchronize(s.cs);
    cudaFreeHost(s.h_syn); cudaFreeHost(s.h_gid); cudaFreeHost(s.h_off); cudaFreeHost(s.h_rid);
    cudaFreeHost(s.h_tsub); cudaFreeHost(s.h_obs); cudaFreeHost(s.h_w); cudaFreeHost(s.h_st);
    cudaFreeHost(s.h_done);
    cudaFree(s.d_syn); cudaFree(s.d_gid); cudaFree(s.d_off);
    cudaFree(s.slabs); cudaFree(s.slabs2); cudaFree(s.queue); cudaFree(s.overflow);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.cs) cudaStreamDestroy(s.cs);
    s = Slot();
}

bool alloc_slot(qec_stream *st, Slot &s) {
    const size_t R = (size_t)st->cap_req, W = (size_t)st->cap_words;
    bool ok = cudaStreamCreateWithFlags(&s.cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaHostAlloc(&s.h_syn, W * 4, cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&s.h_gid, R * 4, cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&s.h_off, R * 8, cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&s.h_rid, R * 8, cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&s.h_tsub, R * 8, cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&s.h_obs, R * 8, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s.h_w, R * 8, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s.h_st, R * 4, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s.h_done, R * 4, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&s.m_obs, s.h_obs, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&s.m_w, s.h_w, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&s.m_st, s.h_st, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&s.m_done, s.h_done, 0) == cudaSuccess &&
              cudaMalloc(&s.d_syn, W * 4) == cudaSuccess && cudaMalloc(&s.d_gid, R * 4) == cudaSuccess &&
              cudaMalloc(&s.d_off, R * 8) == cudaSuccess &&
              cudaMalloc(&s.slabs, (size_t)(st->sb * st->nwarps)) == cudaSuccess &&
              cudaMalloc(&s.slabs2, (size_t)(st->sb2 * st->nwarps2)) == cudaSuccess &&
              cudaMalloc(&s.queue, 4 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&s.overflow, R * 4) == cudaSuccess &&
              // the kernel expects empty (all-ones) table entries and leaves them so
              cudaMemset(s.slabs, 0xff, (size_t)(st->sb * st->nwarps)) == cudaSuccess &&
              cudaMemset(s.slabs2, 0xff, (size_t)(st->sb2 * st->nwarps2)) == cudaSuccess;
    return ok;
}

// Enqueue one micro-batch on its slot's stream (the slot is owned by the dispatcher).
cudaError_t launch_slot(qec_stream *st, Slot &s) {
    cudaError_t e;
    // completion flags cleared before the launch (the launch orders these host
    // writes before the kernel's)
    std::memset(s.h_done, 0, (size_t)s.n * sizeof(int32_t));
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s.pending.resize((size_t)s.n);
    for (int k = 0; k < s.n; k++) s.pending[(size_t)k] = k;
    if ((e = cudaMemcpyAsync(s.d_syn, s.h_syn, (size_t)s.words * 4, cudaMemcpyHostToDevice, s.cs))) return e;
    if ((e = cudaMemcpyAsync(s.d_gid, s.h_gid, (size_t)s.n * 4, cudaMemcpyHostToDevice, s.cs))) return e;
    if ((e = cudaMemcpyAsync(s.d_off, s.h_off, (size_t)s.n * 8, cudaMemcpyHostToDevice, s.cs))) return e;
    if ((e = qec::launch_reset_queue(s.queue, s.cs))) return e;
    qec::BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    {
        std::lock_guard<std::mutex> lk(st->mu);   // the registry only grows, under this lock
        for (size_t i = 0; i < st->views.size(); i++) a.g[i] = st->views[i];
        a.num_graphs = (int)st->views.size();
    }
    a.band_factor = 1;
    a.num_shots = s.n;
    a.max_events = 4000000;
    a.graph_of_shot = s.d_gid;
    a.syn_off = reinterpret_cast<const long long *>(s.d_off);
    a.syn = s.d_syn;
    a.obs_out = reinterpret_cast<unsigned long long *>(s.m_obs);
    a.w_out = reinterpret_cast<long long *>(s.m_w);
    a.st_out = s.m_st;
    a.done = s.m_done;
    a.queue = s.queue;
    a.overflow = s.overflow;
    a.single_shot = -1;
    a.watchdog_ns = 60LL * 1000 * 1000 * 1000;
    a.slabs = s.slabs;
    a.slab_bytes = st->sb;
    a.caps = st->caps;
    a.pass = 0;
    // team size per window: set by qec_set_tuning, else a block of TEAM_BIG
    // warps per window while the micro-batch has at most one window per
    // available block (requests are latency-bound, the GPU has room to spare),
    // one warp per window beyond that
    const qec_tuning tune = qec::current_tuning();
    a.team_split = tune.team_split_events;
    int team = tune.team_warps;
    if (team <= 0) team = s.n <= st->team_blocks ? qec::TEAM_BIG : 1;
    if (team > 1) {
        const int blocks = std::min(s.n, st->nwarps);
        if ((e = qec::launch_batch(a, blocks, 32 * team, s.cs, team))) return e;
    } else {
        const int wpb = 4;
        int warps = std::min(st->nwarps, (s.n + 0));
        warps = (warps + wpb - 1) / wpb * wpb;
        if ((e = qec::launch_batch(a, warps / wpb, 32 * wpb, s.cs))) return e;
    }
    a.slabs = s.slabs2;
    a.slab_bytes = st->sb2;
    a.caps = st->caps2;
    a.pass = 1;
    if ((e = qec::launch_batch(a, st->nwarps2, team > 1 ? 32 * team : 32, s.cs, team))) return e;
    return cudaEventRecord(s.ev, s.cs);
}

void dispatcher(qec_stream *st) {
    cudaSetDevice(st->device);
    std::vector<qec_result> out;
    while (!st->stop.load(std::memory_order_relaxed)) {
        bool busy = false;
        // completions: in-flight slots belong to this thread.  Every window
        // whose flag is set is handed out at once; the slot is reused when the
        // kernel has finished and every window is out (after a failed launch
        // the remaining windows end with QEC_SHOT_INTERNAL).
        int inflight = 0;
        for (int i = 0; i < st->nslots; i++) {
            Slot &s = st->slots[i];
            if (s.state != INFLIGHT) continue;
            const cudaError_t q = cudaEventQuery(s.ev);
            const bool finished = q != cudaErrorNotReady;
            const int64_t t = mono_ns();
            out.clear();
            size_t keep = 0;
            for (size_t j = 0; j < s.pending.size(); j++) {
                const int k = s.pending[j];
                const bool flag = __atomic_load_n(&s.h_done[k], __ATOMIC_ACQUIRE) != 0;
                if (!flag && !finished) { s.pending[keep++] = k; continue; }
                qec_result r;
                r.request_id = s.h_rid[k];
                const bool ok = flag || q == cudaSuccess;
                r.obs = ok ? s.h_obs[k] : 0;
                r.weight = ok ? s.h_w[k] : 0;
                r.status = ok ? s.h_st[k] : QEC_SHOT_INTERNAL;
                r.graph_index = s.h_gid[k];
                r.t_submit_ns = s.h_tsub[k];
                r.t_done_ns = t;
                out.push_back(r);
            }
            s.pending.resize(keep);
            const bool recycle = finished && keep == 0;
            if (!recycle) inflight++;
            if (out.empty() && !recycle) continue;
            std::lock_guard<std::mutex> lk(st->mu);
            if (finished && q != cudaSuccess && st->err.empty()) st->err = cudaGetErrorString(q);
            st->done.insert(st->done.end(), out.begin(), out.end());
            st->admitted -= (int)out.size();
            if (recycle) {
                s.n = 0;
                s.words = 0;
                s.state = IDLE;
            }
            busy = true;
        }
        // launch the filling micro-batch when an in-flight slot is free
        int launch = -1;
        {
            std::lock_guard<std::mutex> lk(st->mu);
            if (st->filling >= 0 && st->slots[st->filling].n > 0 && inflight < st->nslots - 1) {
                launch = st->filling;
                st->slots[launch].state = INFLIGHT;
                st->filling = -1;
            }
            if (st->filling < 0) {
                for (int i = 0; i < st->nslots; i++)
                    if (st->slots[i].state == IDLE) {
                        st->slots[i].state = FILLING;
                        st->filling = i;
                        break;
                    }
            }
        }
        if (launch >= 0) {
            const cudaError_t e = launch_slot(st, st->slots[launch]);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(st->mu);
                if (st->err.empty()) st->err = cudaGetErrorString(e);
            }
            busy = true;
        }
        if (!busy) std::this_thread::yield();
    }
}

}  // namespace

extern "C" {

int qec_stream_create(size_t device_budget_bytes, int32_t max_inflight, qec_stream **out) {
    if (!out) return ferr(QEC_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_inflight < 1) return ferr(QEC_EINVAL, "max_inflight must be >= 1");
    qec_stream *st = new (std::nothrow) qec_stream();
    if (!st) return ferr(QEC_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&st->device) != cudaSuccess) { delete st; return ferr(QEC_ECUDA, "cudaGetDevice failed"); }
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, st->device);
    st->max_inflight = max_inflight;
    st->nwarps = 2 * sms;
    st->nwarps2 = 16;
    st->team_blocks = sms * qec::team_occupancy_blocks(qec::TEAM_BIG);
    st->caps = qec::caps_for_kcap(512, 1);
    st->caps2 = qec::caps_for_kcap(2048, 2);
    st->sb = qec::slab_bytes_for(st->caps);
    st->sb2 = qec::slab_bytes_for(st->caps2);
    st->cap_req = std::min(max_inflight, 1 << 16);
    st->cap_words = std::min<long long>((long long)st->cap_req * QEC_STREAM_MAX_WORDS, 1LL << 22);
    const long long per_slot = st->sb * st->nwarps + st->sb2 * st->nwarps2 + st->cap_words * 4 +
                               (long long)st->cap_req * 48 + 4096;
    const long long n = (long long)device_budget_bytes / per_slot;
    if (n < 2) {
        delete st;
        return ferr(QEC_ENOMEM, "device budget holds fewer than two in-flight slots (" +
                                    std::to_string(per_slot) + " bytes each)");
    }
    st->nslots = (int)std::min<long long>(n, 8);
    st->slots.resize((size_t)st->nslots);
    for (int i = 0; i < st->nslots; i++) {
        if (!alloc_slot(st, st->slots[i])) {
            for (auto &s : st->slots) free_slot(s);
            delete st;
            return ferr(QEC_ENOMEM, "stream slot allocation failed");
        }
    }
    st->slots[0].state = FILLING;
    st->filling = 0;
    st->th = std::thread(dispatcher, st);
    *out = st;
    return QEC_OK;
}

}  // extern "C"

namespace {

// Append one window to the filling micro-batch; the caller holds st->mu.
int submit_locked(qec_stream *st, const qec_graph *g, const uint32_t *syndrome_host, uint64_t request_id,
                  int64_t t_now) {
    if (!g || !syndrome_host) return ferr(QEC_EINVAL, "NULL argument");
    if (!st->err.empty()) return ferr(QEC_ECUDA, "stream failed: " + st->err);
    int gi = -1;
    for (size_t i = 0; i < st->graphs.size(); i++)
        if (st->graphs[i] == g) gi = (int)i;
    if (gi < 0) {
        qec::DGraph view;
        int gdev = -1;
        if (qec::graph_device_view(g, &view, &gdev) != QEC_OK || gdev != st->device)
            return ferr(QEC_EINVAL, "graph lives on another device");
        if (view.words > QEC_STREAM_MAX_WORDS) return ferr(QEC_ERANGE, "window larger than QEC_STREAM_MAX_WORDS");
        if ((int)st->graphs.size() >= QEC_STREAM_MAX_GRAPHS) return ferr(QEC_ERANGE, "too many graphs in one stream");
        st->graphs.push_back(g);
        st->views.push_back(view);
        gi = (int)st->graphs.size() - 1;
    }
    const int words = st->views[(size_t)gi].words;
    if (st->admitted >= st->max_inflight) return QEC_EAGAIN;
    if (st->filling < 0) return QEC_EAGAIN;
    Slot &s = st->slots[st->filling];
    if (s.n >= st->cap_req || s.words + words > st->cap_words) return QEC_EAGAIN;
    std::memcpy(s.h_syn + s.words, syndrome_host, (size_t)words * 4);
    s.h_gid[s.n] = gi;
    s.h_off[s.n] = s.words;
    s.h_rid[s.n] = request_id;
    s.h_tsub[s.n] = t_now;
    s.n++;
    s.words += words;
    st->admitted++;
    return QEC_OK;
}

}  // namespace

extern "C" {

int qec_stream_submit(qec_stream *st, const qec_graph *g, const uint32_t *syndrome_host, uint64_t request_id) {
    if (!st) return ferr(QEC_EINVAL, "NULL stream");
    const int64_t t = mono_ns();
    std::lock_guard<std::mutex> lk(st->mu);
    return submit_locked(st, g, syndrome_host, request_id, t);
}

int qec_stream_submit_many(qec_stream *st, const qec_graph *const *graphs, int32_t num_graphs,
                           const int32_t *graph_of_req, const int64_t *syn_offset_words,
                           const uint32_t *syndromes_host, const uint64_t *request_ids, int32_t n,
                           int32_t *n_accepted) {
    if (!n_accepted) return ferr(QEC_EINVAL, "NULL n_accepted");
    *n_accepted = 0;
    if (n < 0 || (n > 0 && (!st || !graphs || !graph_of_req || !syn_offset_words || !syndromes_host ||
                            !request_ids)))
        return ferr(QEC_EINVAL, "NULL argument");
    const int64_t t = mono_ns();
    std::lock_guard<std::mutex> lk(st->mu);
    for (int32_t i = 0; i < n; i++) {
        const int gi = graph_of_req[i];
        if (gi < 0 || gi >= num_graphs) return ferr(QEC_EINVAL, "graph index out of range");
        const int rc = submit_locked(st, graphs[gi], syndromes_host + syn_offset_words[i], request_ids[i], t);
        if (rc == QEC_EAGAIN) return QEC_OK;
        if (rc != QEC_OK) return rc;
        *n_accepted = i + 1;
    }
    return QEC_OK;
}

int qec_stream_poll(qec_stream *st, qec_result *out, int32_t max, int32_t *n_out) {
    if (!st || !n_out || (max > 0 && !out)) return ferr(QEC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(st->mu);
    int k = 0;
    while (k < max && !st->done.empty()) {
        out[k++] = st->done.front();
        st->done.pop_front();
    }
    *n_out = k;
    if (!st->err.empty()) return ferr(QEC_ECUDA, "stream failed: " + st->err);
    return QEC_OK;
}

int qec_stream_flush(qec_stream *st) {
    if (!st) return ferr(QEC_EINVAL, "NULL stream");
    // every launch ends within the kernels' 60 s watchdog; give up after 10 minutes
    const int64_t t_end = mono_ns() + 600LL * 1000000000LL;
    while (mono_ns() < t_end) {
        {
            std::lock_guard<std::mutex> lk(st->mu);
            if (!st->err.empty()) return ferr(QEC_ECUDA, "stream failed: " + st->err);
            if (st->admitted == 0) return QEC_OK;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return ferr(QEC_ECUDA, "qec_stream_flush timed out");
}

int qec_stream_destroy(qec_stream *st) {
    if (!st) return QEC_OK;
    st->stop.store(true);
    if (st->th.joinable()) st->th.join();
    for (auto &s : st->slots) free_slot(s);
    delete st;
    return QEC_OK;
}

}  // extern "C"
