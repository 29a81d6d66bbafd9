// capi.cpp -- host side of the C ABI declared in include/qec.h.
//
// Graph creation (validation, parallel-edge merging, CSR upload, Algorithm 3
// schedule in exact rational arithmetic), the device workspace and the batch /
// plain launch paths.  Kernels live in decoder.cu.

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "qec_internal.h"

using qec::BatchArgs;
using qec::DGraph;
using qec::SlabCaps;
using qec::Slot;

struct qec_graph {
    int device = -1;
    int n = 0;
    int m = 0;                      // merged edges
    int words = 0;
    int wmax = 0;                   // internal
    int internal_obs = 0;
    int num_levels = 0;
    long long dk[8] = {0}, bk[8] = {0};
    std::vector<int> eu, ev, ew;    // merged edges (host copy)
    std::vector<unsigned long long> eobs;
    int *d_row = nullptr;
    Slot *d_slot = nullptr;
    int *d_seid = nullptr;
    unsigned long long *d_eobs = nullptr;
    int2 *d_eend = nullptr;
    unsigned *d_commit = nullptr;   // commit-region bitmap (sliding windows)
    int components = 0;             // connected components of the detector graph
    long long diam_ub = 0;          // upper bound on detector-detector distances (internal units)
    int upper_single = 0;           // every event above level 1 forms one processing cluster
    qec_params params{};            // Algorithm 3 inputs given at creation
    bool has_params = false;
    DGraph dg{};
};

namespace {

thread_local std::string g_err = "";

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return QEC_ECUDA;
}

// ------------------------------------------------------------ rationals --
// Exact rationals on __int128 with overflow detection, for Algorithm 3.
struct Q {
    __int128 n, d;   // d > 0, gcd(n, d) == 1
};

__int128 gcd128(__int128 a, __int128 b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) { __int128 t = a % b; a = b; b = t; }
    return a ? a : 1;
}

bool mk(__int128 n, __int128 d, Q &out) {
    if (d == 0) return false;
    if (d < 0) { n = -n; d = -d; }
    __int128 g = gcd128(n, d);
    out.n = n / g;
    out.d = d / g;
    return true;
}

bool mul128(__int128 a, __int128 b, __int128 &r) { return !__builtin_mul_overflow(a, b, &r); }
bool add128(__int128 a, __int128 b, __int128 &r) { return !__builtin_add_overflow(a, b, &r); }

bool qadd(Q a, Q b, Q &r) {
    __int128 x, y, z, w;
    if (!mul128(a.n, b.d, x) || !mul128(b.n, a.d, y) || !add128(x, y, z) || !mul128(a.d, b.d, w)) return false;
    return mk(z, w, r);
}
bool qneg(Q a, Q &r) { r.n = -a.n; r.d = a.d; return true; }
bool qsub(Q a, Q b, Q &r) { Q nb; qneg(b, nb); return qadd(a, nb, r); }
bool qmul(Q a, Q b, Q &r) {
    __int128 x, w;
    if (!mul128(a.n, b.n, x) || !mul128(a.d, b.d, w)) return false;
    return mk(x, w, r);
}
bool qdiv(Q a, Q b, Q &r) {
    if (b.n == 0) return false;
    __int128 x, w;
    if (!mul128(a.n, b.d, x) || !mul128(a.d, b.n, w)) return false;
    return mk(x, w, r);
}
// sign of a - b, or 2 on overflow
int qcmp(Q a, Q b) {
    __int128 x, y;
    if (!mul128(a.n, b.d, x) || !mul128(b.n, a.d, y)) return 2;
    return x < y ? -1 : (x > y ? 1 : 0);
}
Q qint(long long v) { return Q{(__int128)v, 1}; }
__int128 qfloor(Q a) {
    __int128 f = a.n / a.d;
    if ((a.n % a.d != 0) && (a.n < 0)) f -= 1;
    return f;
}
__int128 qceil(Q a) { return -qfloor(Q{-a.n, a.d}); }

// Phi_{k+1}(b) = phi - (phi + 2) d / ((phi + 1) d + phi b)
bool big_phi(Q phi, long long d, long long b, Q &out) {
    Q two = qint(2), one = qint(1), dd = qint(d), bb = qint(b);
    Q num, den, t1, t2, frac;
    if (!qadd(phi, two, t1) || !qmul(t1, dd, num)) return false;
    if (!qadd(phi, one, t1) || !qmul(t1, dd, t1) || !qmul(phi, bb, t2) || !qadd(t1, t2, den)) return false;
    if (!qdiv(num, den, frac)) return false;
    return qsub(phi, frac, out);
}

// admissible(b): b >= d, b > 0, phi > 2d/b, Phi(b) >= target.  -1 on overflow.
int admissible(Q phi, long long d, long long b, Q target) {
    if (b < d || b <= 0) return 0;
    Q r;
    if (!qdiv(qint(2 * d), qint(b), r)) return -1;
    int c = qcmp(phi, r);
    if (c == 2) return -1;
    if (c <= 0) return 0;
    Q p;
    if (!big_phi(phi, d, b, p)) return -1;
    c = qcmp(p, target);
    if (c == 2) return -1;
    return c >= 0 ? 1 : 0;
}

// Algorithm 3 (Methods, "Finite-size parameter schedule"), internal units.
// d1c / b1c > 0 replace the level-1 diameter / buffer (b1c must be admissible
// for level 1: b >= d, phi_1 = 1 > 2d/b, Phi_2(b) >= phibar_2); the schedule
// continues from them by the same recursion.
int schedule(int wmax, Q q, Q phimin, long long *dk, long long *bk, int maxlev, long long d1c = 0,
             long long b1c = 0) {
    Q phi = qint(1);
    long long d = d1c > 0 ? d1c : (long long)wmax + 1;
    int lev = 0;
    for (int k = 1; k <= maxlev; k++) {
        // phibar_{k+1} = phimin + (1 - phimin) q^k
        Q qk = qint(1), t, one_m, target;
        bool ok = true;
        for (int i = 0; i < k && ok; i++) ok = qmul(qk, q, qk);
        ok = ok && qsub(qint(1), phimin, one_m) && qmul(one_m, qk, t) && qadd(phimin, t, target);
        if (!ok) break;
        if (qcmp(phi, target) != 1) break;
        // b > 2d / phi
        Q r;
        if (!qdiv(qint(2 * d), phi, r)) break;
        __int128 lo1 = qfloor(r) + 1;
        // Phi(b) >= target  <=>  b >= ((phi + 2) d / (phi - target) - (phi + 1) d) / phi
        Q a1, a2, a3, a4, x;
        if (!qadd(phi, qint(2), a1) || !qmul(a1, qint(d), a1) || !qsub(phi, target, a2) ||
            !qdiv(a1, a2, a3) || !qadd(phi, qint(1), a4) || !qmul(a4, qint(d), a4) ||
            !qsub(a3, a4, x) || !qdiv(x, phi, x))
            break;
        __int128 lo2 = qceil(x);
        __int128 b = d;
        if (lo1 > b) b = lo1;
        if (lo2 > b) b = lo2;
        if (b < 1) b = 1;
        if (b > (__int128)(1LL << 61)) break;
        long long bl = (long long)b;
        if (k == 1 && b1c > 0) {
            if (admissible(phi, d, b1c, target) != 1) break;   // a custom b_1 need not be the smallest
            bl = b1c;
        } else {
            if (admissible(phi, d, bl, target) != 1) break;
            if (bl - 1 >= 1 && admissible(phi, d, bl - 1, target) != 0) break;
        }
        dk[lev] = d;
        bk[lev] = bl;
        lev++;
        Q nphi;
        if (!big_phi(phi, d, bl, nphi)) break;
        phi = nphi;
        __int128 nd = (__int128)3 * d + (__int128)4 * bl + (__int128)2 * wmax;
        if (nd > (__int128)(1LL << 61)) break;
        d = (long long)nd;
    }
    return lev;
}

struct PhysKey {
    int lo, hi, w, idx;
};

// Exact single-source distances over detector-detector slots (boundary
// vertices are leaves, so no path passes through them).
void dijkstra_host(const std::vector<int> &row, const std::vector<Slot> &slots, int src, std::vector<long long> &dist) {
    const long long INF = LLONG_MAX;
    std::fill(dist.begin(), dist.end(), INF);
    using Item = std::pair<long long, int>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    dist[(size_t)src] = 0;
    pq.push({0, src});
    while (!pq.empty()) {
        const Item it = pq.top();
        pq.pop();
        if (it.first != dist[(size_t)it.second]) continue;
        for (int j = row[(size_t)it.second]; j < row[(size_t)it.second + 1]; j++) {
            const Slot sl = slots[(size_t)j];
            if (sl.code < 0) continue;
            const long long nd = it.first + sl.w;
            if (nd < dist[(size_t)sl.code]) {
                dist[(size_t)sl.code] = nd;
                pq.push({nd, sl.code});
            }
        }
    }
}

// Connected components of the detector graph and an upper bound on the
// distance between two detectors of one component: 2 x the eccentricity of a
// central vertex (triangle inequality through it).  Three Dijkstra runs per
// component: from its first vertex v, from the vertex x farthest from v, and
// from the vertex c minimising max(d(v, c), d(x, c)).
void graph_extent(int n, const std::vector<int> &row, const std::vector<Slot> &slots, int &components,
                  long long &diam_ub) {
    std::vector<int> comp((size_t)n, -1);
    std::vector<long long> dv((size_t)n), dx((size_t)n), dc((size_t)n);
    components = 0;
    diam_ub = 0;
    for (int v = 0; v < n; v++) {
        if (comp[(size_t)v] >= 0) continue;
        dijkstra_host(row, slots, v, dv);
        int x = v;
        for (int y = 0; y < n; y++)
            if (dv[(size_t)y] != LLONG_MAX) {
                comp[(size_t)y] = components;
                if (dv[(size_t)y] > dv[(size_t)x]) x = y;
            }
        dijkstra_host(row, slots, x, dx);
        int c = v;
        long long best = LLONG_MAX;
        for (int y = 0; y < n; y++)
            if (comp[(size_t)y] == components) {
                const long long m = std::max(dv[(size_t)y], dx[(size_t)y]);
                if (m < best) { best = m; c = y; }
            }
        dijkstra_host(row, slots, c, dc);
        long long ecc_v = 0, ecc_c = 0;
        for (int y = 0; y < n; y++)
            if (comp[(size_t)y] == components) {
                ecc_v = std::max(ecc_v, dv[(size_t)y]);
                ecc_c = std::max(ecc_c, dc[(size_t)y]);
            }
        diam_ub = std::max(diam_ub, 2 * std::min(ecc_v, ecc_c));
        components++;
    }
}

// ------------------------------------------------------------ workspace --
struct Workspace {
    int device = -1;
    char *slabs = nullptr;
    long long slab_bytes = 0;
    long long nwarps = 0;
    SlabCaps caps{};
    char *slabs2 = nullptr;          // overflow pass
    long long slab_bytes2 = 0;
    long long nwarps2 = 0;
    SlabCaps caps2{};
    unsigned long long *queue = nullptr;
    int *overflow = nullptr;
    int *order = nullptr;          // graph-sorted work order of a mixed batch
    bool fill1 = false, fill2 = false;   // slabs to fill with ones before the next launch
    int *gcnt = nullptr;           // 64 ints: per-graph counts and cursors
    long long overflow_cap = 0;
    cudaEvent_t done = nullptr;
    std::mutex mu;
};

Workspace g_ws[64];
std::mutex g_tune_mu;
qec_tuning g_tune = {4, 0, 1, 0, 4000000, 0, 2048, 1};

void ws_free(Workspace &w) {
    if (w.slabs) cudaFree(w.slabs);
    if (w.slabs2) cudaFree(w.slabs2);
    if (w.queue) cudaFree(w.queue);
    if (w.overflow) cudaFree(w.overflow);
    if (w.order) cudaFree(w.order);
    if (w.gcnt) cudaFree(w.gcnt);
    if (w.done) cudaEventDestroy(w.done);
    w.slabs = w.slabs2 = nullptr;
    w.queue = nullptr;
    w.overflow = nullptr;
    w.order = nullptr;
    w.gcnt = nullptr;
    w.done = nullptr;
    w.slab_bytes = w.slab_bytes2 = 0;
    w.nwarps = w.nwarps2 = 0;
    w.overflow_cap = 0;
}

// Graphs this large are decoded by block-wide teams under the automatic team
// choice (windows of d >= 41).
constexpr int kTeamMidDetectors = 32768;

// Default detection events per main-pass slab: num_detectors / 16, clamped to
// 64 .. 1024, or to 64 .. 4096 when block-wide teams decode a graph of at least
// kTeamMidDetectors detectors (those launches hold one slab per resident block
// only; a d = 51 window holds ~1,200 events at p = 0.003 and ~1,900 at
// p = 0.005; past kcap a shot goes to the overflow pass, which has one team
// per SM).
int kcap_for(int nmax, const qec_tuning &t, bool blocks) {
    if (t.kcap > 0) return std::min(t.kcap, std::max(1, nmax));
    int k = nmax / 16;
    k = std::max(64, std::min(blocks && nmax >= kTeamMidDetectors ? 4096 : 1024, k));
    return std::min(k, std::max(nmax, 1));
}

// Every capacity of `have` at least that of `need`: a slab laid out for
// `have` serves the request (capacities change no result, only which shots
// run out of room).
bool caps_cover(const SlabCaps &have, const SlabCaps &need) {
    return have.kc >= need.kc && have.hc >= need.hc && have.ec >= need.ec && have.wc >= need.wc &&
           have.phc >= need.phc && have.nc >= need.nc && have.cc >= need.cc && have.wcap >= need.wcap;
}

// Make sure the workspace of `dev` fits the request; may synchronise the device.
// Unless `exact` (a slab size set through qec_set_tuning), a slab layout that
// already covers the request is kept as it is (no new allocation and no
// refill), so alternating batch shapes reuse the largest.
int ws_ensure(Workspace &w, int dev, SlabCaps caps, long long nwarps, SlabCaps caps2, long long nwarps2,
              long long nshots, bool exact) {
    w.device = dev;
    if (!exact && w.slabs && nwarps <= w.nwarps && caps_cover(w.caps, caps)) caps = w.caps;
    if (!exact && w.slabs2 && nwarps2 <= w.nwarps2 && caps_cover(w.caps2, caps2)) caps2 = w.caps2;
    const long long sb = qec::slab_bytes_for(caps);
    const long long sb2 = qec::slab_bytes_for(caps2);
    cudaError_t e;
    if (!w.done) {
        e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        e = cudaEventRecord(w.done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    const bool grow1 = sb * nwarps > w.slab_bytes * w.nwarps || sb != w.slab_bytes || nwarps > w.nwarps;
    const bool grow2 = sb2 * nwarps2 > w.slab_bytes2 * w.nwarps2 || sb2 != w.slab_bytes2 || nwarps2 > w.nwarps2;
    const bool grow3 = nshots > w.overflow_cap || !w.queue;
    if (grow1 || grow2 || grow3) {
        e = cudaEventSynchronize(w.done);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    }
    // the kernel expects every explored / pair table entry to be all ones on
    // entry and leaves it so; a new allocation or a new slab layout is filled
    if (grow1 || std::memcmp(&w.caps, &caps, sizeof(caps)) != 0) w.fill1 = true;
    if (grow2 || std::memcmp(&w.caps2, &caps2, sizeof(caps2)) != 0) w.fill2 = true;
    if (grow1) {
        if (w.slabs) cudaFree(w.slabs);
        w.slabs = nullptr;
        e = cudaMalloc(&w.slabs, (size_t)(sb * nwarps));
        if (e != cudaSuccess) { w.slab_bytes = 0; w.nwarps = 0; return fail(QEC_ENOMEM, "workspace allocation failed"); }
        w.slab_bytes = sb;
        w.nwarps = nwarps;
    }
    w.caps = caps;
    if (grow2) {
        if (w.slabs2) cudaFree(w.slabs2);
        w.slabs2 = nullptr;
        e = cudaMalloc(&w.slabs2, (size_t)(sb2 * nwarps2));
        if (e != cudaSuccess) { w.slab_bytes2 = 0; w.nwarps2 = 0; return fail(QEC_ENOMEM, "workspace allocation failed"); }
        w.slab_bytes2 = sb2;
        w.nwarps2 = nwarps2;
    }
    w.caps2 = caps2;
    if (grow3) {
        if (!w.queue) {
            e = cudaMalloc(&w.queue, 4 * sizeof(unsigned long long));
            if (e != cudaSuccess) return fail(QEC_ENOMEM, "workspace allocation failed");
        }
        if (w.overflow) cudaFree(w.overflow);
        if (w.order) cudaFree(w.order);
        w.overflow = nullptr;
        w.order = nullptr;
        long long cap = std::max<long long>(nshots, 1024);
        e = cudaMalloc(&w.overflow, (size_t)cap * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&w.order, (size_t)cap * sizeof(int));
        if (e == cudaSuccess && !w.gcnt) e = cudaMalloc(&w.gcnt, 64 * sizeof(int));
        if (e != cudaSuccess) { w.overflow_cap = 0; return fail(QEC_ENOMEM, "workspace allocation failed"); }
        w.overflow_cap = cap;
    }
    return QEC_OK;
}

// Whether the workspace already holds this request as it stands (no growth,
// same slab layouts, nothing left to fill): the condition for decoding inside
// a stream capture, where nothing may be allocated or synchronised.
bool ws_fits(const Workspace &w, const SlabCaps &caps, long long nwarps, const SlabCaps &caps2, long long nwarps2,
             long long nshots, bool exact) {
    if (!w.done || !w.queue || !w.slabs || !w.slabs2 || w.fill1 || w.fill2) return false;
    if (nwarps > w.nwarps || nwarps2 > w.nwarps2 || nshots > w.overflow_cap) return false;
    if (exact)
        return std::memcmp(&w.caps, &caps, sizeof(caps)) == 0 && std::memcmp(&w.caps2, &caps2, sizeof(caps2)) == 0;
    return caps_cover(w.caps, caps) && caps_cover(w.caps2, caps2);
}

int sm_count(int dev) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

}  // namespace

int qec::graph_device_view(const qec_graph *g, DGraph *out, int *device) {
    if (!g || !out || !device) return QEC_EINVAL;
    *out = g->dg;
    *device = g->device;
    return QEC_OK;
}

qec_tuning qec::current_tuning() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

int qec::set_last_error(int code, const char *msg) {
    g_err = msg ? msg : "";
    return code;
}

extern "C" {

const char *qec_last_error(void) { return g_err.c_str(); }

const char *qec_version(void) { return "qec-sparse-blossom-gb300 0.1 (sm_103a)"; }

int qec_schedule(int32_t wmax_internal, const qec_params *params, int64_t *d_k, int64_t *b_k,
                 int32_t max_levels) {
    if (wmax_internal < 1 || !d_k || !b_k || max_levels < 1 || max_levels > 64)
        return fail(QEC_EINVAL, "bad schedule arguments");
    Q q = {1, 10}, phimin = {1, 100};
    long long d1c = 0, b1c = 0;
    if (params) {
        if (params->q_den <= 0 || params->phi_den <= 0 || params->q_num <= 0 || params->phi_num <= 0 ||
            params->q_num >= params->q_den || params->phi_num >= params->phi_den)
            return fail(QEC_EINVAL, "params must be fractions in (0, 1)");
        if (params->d1 < 0 || params->b1 < 0) return fail(QEC_EINVAL, "negative level-1 override");
        mk(params->q_num, params->q_den, q);
        mk(params->phi_num, params->phi_den, phimin);
        d1c = params->d1;
        b1c = params->b1;
    }
    std::vector<long long> dk((size_t)max_levels), bk((size_t)max_levels);
    const int lev = schedule(wmax_internal, q, phimin, dk.data(), bk.data(), max_levels, d1c, b1c);
    for (int i = 0; i < lev; i++) { d_k[i] = dk[i]; b_k[i] = bk[i]; }
    return lev >= 1 ? lev : fail(QEC_EINVAL, "no admissible level-1 parameters");
}

int qec_graph_create(const qec_graph_desc *desc, qec_graph **out) {
    if (!out) return fail(QEC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(QEC_EINVAL, "desc is NULL");
    const int n = desc->num_detectors, m = desc->num_edges;
    if (n < 1 || n > (1 << 26)) return fail(QEC_ERANGE, "num_detectors out of range");
    if (m < 0 || m > (1 << 28)) return fail(QEC_ERANGE, "num_edges out of range");
    if (desc->num_observables < 0 || desc->num_observables > QEC_MAX_OBSERVABLES)
        return fail(QEC_EINVAL, "num_observables out of range");
    if (m > 0 && (!desc->u || !desc->v || !desc->w || !desc->obs)) return fail(QEC_EINVAL, "edge array is NULL");
    Q q = {1, 10}, phimin = {1, 100};
    long long d1c = 0, b1c = 0;
    if (desc->params) {
        const qec_params *p = desc->params;
        if (p->q_den <= 0 || p->phi_den <= 0 || p->q_num <= 0 || p->phi_num <= 0 || p->q_num >= p->q_den ||
            p->phi_num >= p->phi_den)
            return fail(QEC_EINVAL, "params must be fractions in (0, 1)");
        if (p->d1 < 0 || p->b1 < 0) return fail(QEC_EINVAL, "negative level-1 override");
        mk(p->q_num, p->q_den, q);
        mk(p->phi_num, p->phi_den, phimin);
        d1c = p->d1;
        b1c = p->b1;
    }
    const unsigned long long obs_mask =
        desc->num_observables >= 64 ? ~0ull : ((1ull << desc->num_observables) - 1ull);
    std::vector<PhysKey> keys((size_t)m);
    for (int i = 0; i < m; i++) {
        const int a = desc->u[i], b = desc->v[i], w = desc->w[i];
        if (a < 0 || a >= n || b >= n || a == b) return fail(QEC_EINVAL, "edge endpoint out of range or self loop");
        if (w <= 0 || w > (1 << 20)) return fail(QEC_EINVAL, "edge weight must be in 1 .. 2^20");
        if (desc->obs[i] & ~obs_mask) return fail(QEC_EINVAL, "observable bit beyond num_observables");
        if (b < 0) keys[i] = PhysKey{a, INT32_MAX, w, i};
        else keys[i] = PhysKey{std::min(a, b), std::max(a, b), w, i};
    }
    std::sort(keys.begin(), keys.end(), [](const PhysKey &x, const PhysKey &y) {
        if (x.lo != y.lo) return x.lo < y.lo;
        if (x.hi != y.hi) return x.hi < y.hi;
        if (x.w != y.w) return x.w < y.w;
        return x.idx < y.idx;
    });
    qec_graph *g = new (std::nothrow) qec_graph();
    if (!g) return fail(QEC_ENOMEM, "host allocation failed");
    for (int i = 0; i < m; i++) {
        if (i > 0 && keys[i].lo == keys[i - 1].lo && keys[i].hi == keys[i - 1].hi) continue;
        g->eu.push_back(keys[i].lo);
        g->ev.push_back(keys[i].hi == INT32_MAX ? -1 : keys[i].hi);
        g->ew.push_back(2 * keys[i].w);
        g->eobs.push_back(desc->obs[keys[i].idx]);
    }
    if (desc->params) { g->params = *desc->params; g->has_params = true; }
    g->n = n;
    g->m = (int)g->eu.size();
    g->words = ((n + 31) / 32 + 3) / 4 * 4;
    for (int e = 0; e < g->m; e++) {
        g->wmax = std::max(g->wmax, g->ew[e]);
        if (g->ev[e] >= 0 && g->eobs[e] != 0) g->internal_obs = 1;
    }
    if ((long long)g->wmax * (long long)n > (1LL << 30)) {
        delete g;
        return fail(QEC_ERANGE, "largest weight x detectors exceeds 2^30 (distances are int32)");
    }
    g->num_levels = schedule(g->wmax, q, phimin, g->dk, g->bk, 8, d1c, b1c);
    if (g->num_levels < 1) {
        delete g;
        return fail(QEC_EINVAL, "Algorithm 3 schedule has no admissible level-1 parameters");
    }
    // CSR: slots of each detector in merged-edge order
    std::vector<int> row((size_t)n + 1, 0);
    for (int e = 0; e < g->m; e++) {
        row[g->eu[e] + 1]++;
        if (g->ev[e] >= 0) row[g->ev[e] + 1]++;
    }
    for (int x = 0; x < n; x++) row[x + 1] += row[x];
    std::vector<Slot> slots((size_t)row[n] + 1);
    std::vector<int> seid((size_t)row[n] + 1, -1);
    std::vector<int> fill((size_t)n, 0);
    std::vector<int2> eend((size_t)g->m + 1);
    for (int e = 0; e < g->m; e++) {
        const int a = g->eu[e], b = g->ev[e];
        const int ja = row[a] + fill[a]++;
        slots[ja] = Slot{b >= 0 ? b : -1 - e, g->ew[e]};
        seid[ja] = e;
        if (b >= 0) {
            const int jb = row[b] + fill[b]++;
            slots[jb] = Slot{a, g->ew[e]};
            seid[jb] = e;
        }
        eend[e] = make_int2(a, g->ew[e]);
    }
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) { delete g; return cuda_fail(ce, "cudaGetDevice"); }
    const size_t nslots = (size_t)row[n] + 1, ne = (size_t)g->m + 1;
    ce = cudaMalloc(&g->d_row, sizeof(int) * ((size_t)n + 1));
    if (ce == cudaSuccess) ce = cudaMalloc(&g->d_slot, sizeof(Slot) * nslots);
    if (ce == cudaSuccess) ce = cudaMalloc(&g->d_eobs, sizeof(unsigned long long) * ne);
    if (ce == cudaSuccess) ce = cudaMalloc(&g->d_eend, sizeof(int2) * ne);
    if (ce == cudaSuccess) ce = cudaMalloc(&g->d_seid, sizeof(int) * nslots);
    if (ce != cudaSuccess) { qec_graph_destroy(g); return fail(QEC_ENOMEM, "device allocation failed"); }
    std::vector<unsigned long long> eo(g->eobs);
    eo.push_back(0);
    ce = cudaMemcpy(g->d_row, row.data(), sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(g->d_slot, slots.data(), sizeof(Slot) * nslots, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(g->d_eobs, eo.data(), sizeof(unsigned long long) * ne, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(g->d_eend, eend.data(), sizeof(int2) * ne, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(g->d_seid, seid.data(), sizeof(int) * nslots, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) { qec_graph_destroy(g); return cuda_fail(ce, "cudaMemcpy"); }
    DGraph &d = g->dg;
    d.n = n;
    d.words = g->words;
    d.wmax = g->wmax;
    d.d1 = (int)std::min<long long>(g->dk[0], INT32_MAX / 4);
    d.b1 = (int)std::min<long long>(g->bk[0], INT32_MAX / 4);
    d.internal_obs = g->internal_obs;
    {
        long long wmin = LLONG_MAX;
        for (int e = 0; e < g->m; e++) wmin = std::min<long long>(wmin, g->ew[e]);
        d.hop2 = (g->m > 0 && 3 * wmin > (long long)d.b1) ? 1 : 0;
        d.wmin = g->m > 0 ? (int)std::min<long long>(wmin, INT32_MAX / 4) : 1;
    }
    // Algorithm 1 above level 1: with one connected component and b_2 at least
    // the distance bound, every residual event links to every other at level
    // 2 (and at every later level, b_k grows with k), so all of them form one
    // component at each level until it is accepted (d_k and b_k grow without
    // bound under Algorithm 3's recursion, so it is, unless its parity can never
    // be met).  Then the events left after level 1 form exactly one processing
    // cluster.  b_2 is taken as b_1 when the schedule stored only one level
    // (b_k increases with k, so this only errs on the safe side).
    graph_extent(n, row, slots, g->components, g->diam_ub);
    {
        const long long b2 = g->num_levels >= 2 ? g->bk[1] : g->bk[0];
        g->upper_single = (g->components == 1 && b2 >= g->diam_ub) ? 1 : 0;
    }
    d.row = g->d_row;
    d.slot = g->d_slot;
    d.eobs = g->d_eobs;
    d.eend = g->d_eend;
    d.seid = g->d_seid;
    *out = g;
    return QEC_OK;
}

int qec_graph_create_window(const qec_graph *stream, int32_t first_detector, int32_t num_detectors,
                            const qec_params *params, qec_graph **out) {
    if (!out) return fail(QEC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!stream) return fail(QEC_EINVAL, "stream graph is NULL");
    if (first_detector < 0 || num_detectors < 1 || (long long)first_detector + num_detectors > stream->n)
        return fail(QEC_ERANGE, "window detector range outside the stream graph");
    const int lo = first_detector, hi = first_detector + num_detectors;
    // induced subgraph: merged edges with every detector endpoint inside the
    // window, renumbered from 0 in the same order (the stream graph has no
    // parallel edges left, so merging the window again changes nothing)
    std::vector<int> u, v, w;
    std::vector<uint64_t> o;
    for (int e = 0; e < stream->m; e++) {
        const int a = stream->eu[e], b = stream->ev[e];
        if (a < lo || a >= hi || (b >= 0 && (b < lo || b >= hi))) continue;
        u.push_back(a - lo);
        v.push_back(b >= 0 ? b - lo : -1);
        w.push_back(stream->ew[e] / 2);   // internal weights are twice the integer weights
        o.push_back(stream->eobs[e]);
    }
    qec_graph_desc d;
    std::memset(&d, 0, sizeof(d));
    d.num_detectors = num_detectors;
    d.num_edges = (int)u.size();
    d.num_observables = QEC_MAX_OBSERVABLES;   // masks were validated when the stream graph was created
    d.u = u.data();
    d.v = v.data();
    d.w = w.data();
    d.obs = o.data();
    d.params = params ? params : (stream->has_params ? &stream->params : nullptr);
    return qec_graph_create(&d, out);
}

int qec_graph_destroy(qec_graph *g) {
    if (!g) return QEC_OK;
    if (g->d_row) cudaFree(g->d_row);
    if (g->d_slot) cudaFree(g->d_slot);
    if (g->d_eobs) cudaFree(g->d_eobs);
    if (g->d_eend) cudaFree(g->d_eend);
    if (g->d_seid) cudaFree(g->d_seid);
    if (g->d_commit) cudaFree(g->d_commit);
    delete g;
    return QEC_OK;
}

int qec_graph_set_commit_region(qec_graph *g, const uint32_t *detector_bitmap) {
    if (!g) return fail(QEC_EINVAL, "NULL graph");
    cudaError_t ce;
    if (!detector_bitmap) {
        if (g->d_commit) {
            ce = cudaDeviceSynchronize();   // no decode may still read it
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaDeviceSynchronize");
            cudaFree(g->d_commit);
        }
        g->d_commit = nullptr;
        g->dg.commit = nullptr;
        return QEC_OK;
    }
    std::vector<unsigned> bits((size_t)g->words, 0u);
    for (int i = 0; i < g->words; i++) bits[(size_t)i] = detector_bitmap[i];
    if (g->n % 32) bits[(size_t)(g->n / 32)] &= (1u << (g->n % 32)) - 1u;   // detectors only
    for (int i = g->n / 32 + (g->n % 32 ? 1 : 0); i < g->words; i++) bits[(size_t)i] = 0u;
    if (!g->d_commit) {
        ce = cudaMalloc(&g->d_commit, sizeof(unsigned) * (size_t)g->words);
        if (ce != cudaSuccess) { g->d_commit = nullptr; return fail(QEC_ENOMEM, "cudaMalloc"); }
    }
    ce = cudaMemcpy(g->d_commit, bits.data(), sizeof(unsigned) * (size_t)g->words, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemcpy");
    g->dg.commit = g->d_commit;
    return QEC_OK;
}

int qec_graph_get_info(const qec_graph *g, qec_graph_info *out) {
    if (!g || !out) return fail(QEC_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->num_detectors = g->n;
    out->num_merged_edges = g->m;
    out->words_per_shot = g->words;
    out->wmax_internal = g->wmax;
    out->num_levels = g->num_levels;
    for (int i = 0; i < g->num_levels && i < 8; i++) { out->d_k[i] = g->dk[i]; out->b_k[i] = g->bk[i]; }
    out->device = g->device;
    out->has_internal_obs = g->internal_obs;
    out->components = g->components;
    out->distance_bound = g->diam_ub;
    out->upper_single_cluster = g->upper_single;
    return QEC_OK;
}

int qec_graph_merged_edges(const qec_graph *g, int32_t *u, int32_t *v, int32_t *w, uint64_t *obs) {
    if (!g) return fail(QEC_EINVAL, "graph is NULL");
    for (int e = 0; e < g->m; e++) {
        if (u) u[e] = g->eu[e];
        if (v) v[e] = g->ev[e];
        if (w) w[e] = g->ew[e];
        if (obs) obs[e] = g->eobs[e];
    }
    return QEC_OK;
}

int qec_set_tuning(const qec_tuning *t) {
    if (!t) return fail(QEC_EINVAL, "NULL tuning");
    if (t->warps_per_block > 32 || t->blocks_per_sm > 64 || t->band_factor > 64 || t->kcap > (1 << 18))
        return fail(QEC_EINVAL, "tuning value out of range");
    if (t->team_warps > 0 && t->team_warps != 1 && t->team_warps != qec::TEAM_MID && t->team_warps != qec::TEAM_BIG)
        return fail(QEC_EINVAL, "team_warps must be 1, 4 or 16 (0 keeps, negative = automatic)");
    static const qec_tuning defaults = {4, 0, 1, 0, 4000000, 0, 2048, 1};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto pick = [](auto v, auto cur, auto def) { return v > 0 ? v : (v < 0 ? def : cur); };
    g_tune.warps_per_block = pick(t->warps_per_block, g_tune.warps_per_block, defaults.warps_per_block);
    g_tune.blocks_per_sm = pick(t->blocks_per_sm, g_tune.blocks_per_sm, defaults.blocks_per_sm);
    g_tune.band_factor = pick(t->band_factor, g_tune.band_factor, defaults.band_factor);
    g_tune.kcap = pick(t->kcap, g_tune.kcap, defaults.kcap);
    g_tune.max_events = pick(t->max_events, g_tune.max_events, defaults.max_events);
    g_tune.team_warps = pick(t->team_warps, g_tune.team_warps, defaults.team_warps);
    g_tune.team_min_detectors = pick(t->team_min_detectors, g_tune.team_min_detectors, defaults.team_min_detectors);
    // team_split_events: 0 keeps, negative restores the default, and a value
    // of 1 means every shot goes to the whole team
    g_tune.team_split_events = pick(t->team_split_events, g_tune.team_split_events, defaults.team_split_events);
    return QEC_OK;
}

int qec_get_tuning(qec_tuning *t) {
    if (!t) return fail(QEC_EINVAL, "NULL tuning");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *t = g_tune;
    return QEC_OK;
}

int qec_release_workspace(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(QEC_EINVAL, "device index");
    Workspace &w = g_ws[dev];
    std::lock_guard<std::mutex> lk(w.mu);
    if (w.done) cudaEventSynchronize(w.done);
    ws_free(w);
    return QEC_OK;
}

static int decode_common(const qec_graph *const *graphs, int32_t num_graphs, const int32_t *graph_of_shot,
                         const int64_t *syn_offset_words, const uint32_t *syndromes, int64_t num_shots,
                         uint64_t *obs_out, int64_t *weight_out, int32_t *status_out, qec_cuda_stream stream,
                         bool plain, int32_t mode = QEC_MODE_HIERARCHICAL, int32_t *diag_out = nullptr,
                         uint64_t *commit_obs = nullptr, uint32_t *carry_out = nullptr) {
    if (num_shots < 0) return fail(QEC_EINVAL, "num_shots < 0");
    if (mode != QEC_MODE_HIERARCHICAL && mode != QEC_MODE_GLOBAL) return fail(QEC_EINVAL, "unknown mode");
    const bool window = carry_out != nullptr;
    if (num_shots == 0) return QEC_OK;
    if (!graphs || num_graphs < 1 || num_graphs > QEC_MAX_GRAPHS_PER_BATCH)
        return fail(QEC_EINVAL, "num_graphs out of range");
    if (!syndromes || !status_out || (window ? !commit_obs : (!obs_out || !weight_out)))
        return fail(QEC_EINVAL, "NULL buffer");
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(QEC_EINVAL, "device index");
    int nmax = 1;
    for (int i = 0; i < num_graphs; i++) {
        if (!graphs[i]) return fail(QEC_EINVAL, "NULL graph");
        if (graphs[i]->device != dev) return fail(QEC_EINVAL, "graph lives on another device");
        if (window && !graphs[i]->d_commit) return fail(QEC_EINVAL, "graph has no commit region");
        nmax = std::max(nmax, graphs[i]->n);
    }
    qec_tuning tune;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune = g_tune;
    }
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int sms = sm_count(dev);
    const int wpb = std::max(1, std::min(tune.warps_per_block, qec::max_block_threads() / 32));
    int bps = tune.blocks_per_sm;
    if (bps <= 0) bps = qec::occupancy_blocks(32 * wpb);
    // team size: warps that decode one shot together (the sliding-window
    // kernel is compiled for one warp and for TEAM_BIG warps per shot)
    // automatic choice for a large graph: one 16-warp block per shot when the
    // batch has at most one shot per SM; 4-warp blocks for graphs of at least
    // kTeamMidDetectors detectors (windows of d >= 41: on a GB300 4-warp blocks
    // decoded 2,000 - 4,000 d = 41 windows at p = 0.003 1.6 - 1.9x faster than
    // one warp per window, 3,000 d = 51 windows 2.0x, and lost 18 % only at
    // d = 41, p = 0.001) or while the batch has fewer shots than half the
    // resident one-warp teams (a shot per warp would leave most of the GPU
    // idle); else one warp per shot
    int team = tune.team_warps;
    if (team <= 0) {
        team = 1;
        if (!plain && nmax >= tune.team_min_detectors) {
            const long long resident = (long long)sms * bps * wpb;
            if (num_shots <= sms) team = qec::TEAM_BIG;
            else if (nmax >= kTeamMidDetectors || num_shots * 2 < resident) team = qec::TEAM_MID;
        }
    }
    if (window && team == qec::TEAM_MID) team = 1;
    const int kcap = kcap_for(nmax, tune, team > 1 && !plain);
    SlabCaps caps = qec::caps_for_kcap(kcap);
    // overflow slabs: four times the events (a default capacity above 1,024
    // keeps the overflow slabs at 4,096 events, as with a 1,024 main pass)
    const int kcap2 = (tune.kcap > 0 || kcap <= 1024) ? std::min(nmax, 4 * kcap) : std::min(nmax, 4096);
    SlabCaps caps2 = qec::caps_for_kcap(std::max(kcap, kcap2), 3);
    int wmax_words = 0;
    for (int i = 0; i < num_graphs; i++) wmax_words = std::max(wmax_words, graphs[i]->words);
    caps.wcap = std::max(caps.wcap, wmax_words);
    caps2.wcap = std::max(caps2.wcap, wmax_words);
    // slabs: one per warp of the main pass (one warp per shot) or one per
    // resident block (one block per shot); the overflow pass has one per SM
    long long nwarps = plain ? 1 : (long long)sms * bps * wpb;
    long long nteams = nwarps;
    if (team > 1 && !plain) {
        nteams = std::min<long long>((long long)sms * qec::team_occupancy_blocks(team), std::max<long long>(num_shots, 1));
        // slabs for every resident one-warp team (so that a one-warp call
        // after this one reuses them), except for the largest graphs, whose
        // slabs are big: there only the blocks launched get one
        nwarps = nmax >= kTeamMidDetectors ? nteams : std::max(nwarps, nteams);
    }
    long long nwarps2 = plain ? 1 : (long long)sms;
    if (plain) caps = caps2;
    Workspace &w = g_ws[dev];
    std::lock_guard<std::mutex> lk(w.mu);
    // inside a stream capture the workspace must already fit (a call of the
    // same shape outside capture sizes and fills it), and the workspace event
    // is neither waited on nor recorded: the captured graph's replays are
    // ordered by the caller
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (capturing) {
        if (!ws_fits(w, caps, nwarps, caps2, nwarps2, plain ? 1 : num_shots, tune.kcap > 0))
            return fail(QEC_EINVAL, "stream capture needs a prior uncaptured call of the same shape (workspace not ready)");
    } else {
        int rc = ws_ensure(w, dev, caps, nwarps, caps2, nwarps2, plain ? 1 : num_shots, tune.kcap > 0);
        if (rc != QEC_OK) return rc;
        ce = cudaStreamWaitEvent(s, w.done, 0);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamWaitEvent");
    }
    if (w.fill1) {
        ce = cudaMemsetAsync(w.slabs, 0xff, (size_t)(w.slab_bytes * w.nwarps), s);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemsetAsync");
        w.fill1 = false;
    }
    if (w.fill2) {
        ce = cudaMemsetAsync(w.slabs2, 0xff, (size_t)(w.slab_bytes2 * w.nwarps2), s);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemsetAsync");
        w.fill2 = false;
    }
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int i = 0; i < num_graphs; i++) a.g[i] = graphs[i]->dg;
    a.num_graphs = num_graphs;
    a.band_factor = std::max(1, tune.band_factor);
    a.num_shots = num_shots;
    a.max_events = tune.max_events > 0 ? tune.max_events : 4000000;
    a.graph_of_shot = graph_of_shot;
    a.syn_off = reinterpret_cast<const long long *>(syn_offset_words);
    a.syn = syndromes;
    a.obs_out = reinterpret_cast<unsigned long long *>(obs_out);
    a.w_out = reinterpret_cast<long long *>(weight_out);
    a.st_out = status_out;
    a.queue = w.queue;
    a.overflow = w.overflow;
    a.watchdog_ns = 60LL * 1000 * 1000 * 1000;
    a.mode = mode;
    a.diag_out = diag_out;
    a.cobs = reinterpret_cast<unsigned long long *>(commit_obs);
    a.carry = carry_out;
    a.team_split = tune.team_split_events;
    if (plain) {
        a.slabs = w.slabs;
        a.slab_bytes = w.slab_bytes;
        a.caps = w.caps;
        a.pass = 0;
        for (int64_t shot = 0; shot < num_shots; shot++) {
            a.single_shot = shot;
            ce = qec::launch_batch(a, 1, 32, s, team);
            if (ce != cudaSuccess) return cuda_fail(ce, "kernel launch");
        }
    } else {
        a.single_shot = -1;
        ce = qec::launch_reset_queue(w.queue, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemsetAsync");
        if (num_graphs > 1 && graph_of_shot) {
            // shots grouped by graph, largest graphs first, so concurrent warps
            // share one graph's lines in cache and the longest shots do not trail
            int gorder[QEC_MAX_GRAPHS_PER_BATCH];
            for (int i = 0; i < num_graphs; i++) gorder[i] = i;
            std::stable_sort(gorder, gorder + num_graphs,
                             [&](int x, int y) { return graphs[x]->n > graphs[y]->n; });
            ce = qec::launch_graph_sort(graph_of_shot, num_shots, num_graphs, gorder, w.gcnt, w.order, s);
            if (ce != cudaSuccess) return cuda_fail(ce, "graph sort launch");
            a.order = w.order;
        }
        a.slabs = w.slabs;
        a.slab_bytes = w.slab_bytes;
        a.caps = w.caps;
        a.pass = 0;
        if (team > 1) ce = qec::launch_batch(a, (int)nteams, 32 * team, s, team);
        else ce = qec::launch_batch(a, (int)(nwarps / wpb), 32 * wpb, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "kernel launch");
        a.slabs = w.slabs2;
        a.slab_bytes = w.slab_bytes2;
        a.caps = w.caps2;
        a.pass = 1;
        ce = qec::launch_batch(a, (int)nwarps2, team > 1 ? 32 * team : 32, s, team);
        if (ce != cudaSuccess) return cuda_fail(ce, "kernel launch");
    }
    if (!capturing) {
        ce = cudaEventRecord(w.done, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventRecord");
    }
    return QEC_OK;
}

int qec_decode_batch(const qec_graph *const *graphs, int32_t num_graphs, const int32_t *graph_of_shot,
                     const int64_t *syn_offset_words, const uint32_t *syndromes, int64_t num_shots,
                     uint64_t *obs_out, int64_t *weight_out, int32_t *status_out, qec_cuda_stream stream) {
    return decode_common(graphs, num_graphs, graph_of_shot, syn_offset_words, syndromes, num_shots, obs_out,
                         weight_out, status_out, stream, false);
}

int qec_decode_batch_ex(const qec_graph *const *graphs, int32_t num_graphs, const int32_t *graph_of_shot,
                        const int64_t *syn_offset_words, const uint32_t *syndromes, int64_t num_shots, int32_t mode,
                        uint64_t *obs_out, int64_t *weight_out, int32_t *status_out, int32_t *diag_out,
                        qec_cuda_stream stream) {
    return decode_common(graphs, num_graphs, graph_of_shot, syn_offset_words, syndromes, num_shots, obs_out,
                         weight_out, status_out, stream, false, mode, diag_out);
}

int qec_decode_window_batch(const qec_graph *const *graphs, int32_t num_graphs, const int32_t *graph_of_shot,
                            const int64_t *syn_offset_words, const uint32_t *syndromes, int64_t num_shots,
                            uint64_t *commit_obs_inout, uint32_t *carry_out, int32_t *status_inout,
                            qec_cuda_stream stream) {
    if (!carry_out) return fail(QEC_EINVAL, "NULL buffer");
    return decode_common(graphs, num_graphs, graph_of_shot, syn_offset_words, syndromes, num_shots, nullptr,
                         nullptr, status_inout, stream, false, QEC_MODE_HIERARCHICAL, nullptr, commit_obs_inout,
                         carry_out);
}

int qec_window_assemble(const uint32_t *stream_rows, int64_t stream_words, int64_t bit_begin, int32_t nbits,
                        const uint32_t *carry_rows, int64_t carry_words, int64_t carry_bit_begin,
                        int32_t carry_bits, uint32_t *window_rows, int64_t window_words, int64_t num_rows,
                        qec_cuda_stream stream) {
    if (num_rows < 0 || stream_words < 0 || window_words < 0 || bit_begin < 0 || nbits < 0 ||
        (carry_rows && (carry_words <= 0 || carry_bit_begin < 0 || carry_bits < 0)))
        return fail(QEC_EINVAL, "negative size");
    if (num_rows == 0 || window_words == 0) return QEC_OK;
    if (!stream_rows || !window_rows) return fail(QEC_EINVAL, "NULL buffer");
    if ((long long)nbits > window_words * 32 || (carry_rows && (long long)carry_bits > window_words * 32))
        return fail(QEC_ERANGE, "window row too short");
    const cudaError_t ce = qec::launch_window_assemble(stream_rows, stream_words, bit_begin, nbits, carry_rows,
                                                       carry_words, carry_bit_begin, carry_bits, window_rows,
                                                       window_words, num_rows,
                                                       reinterpret_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) return cuda_fail(ce, "window assemble launch");
    return QEC_OK;
}

int qec_decode_plain(const qec_graph *g, const uint32_t *syndromes, int64_t num_shots, uint64_t *obs_out,
                     int64_t *weight_out, int32_t *status_out, qec_cuda_stream stream) {
    const qec_graph *gs[1] = {g};
    return decode_common(gs, 1, nullptr, nullptr, syndromes, num_shots, obs_out, weight_out, status_out, stream,
                         true);
}

}  // extern "C"
