// decoder.cu -- parallel sparse-blossom decoder for sm_103a.
//
// A team of threads decodes one shot end to end, and a persistent grid of
// teams pulls shots from a device work counter.  A team is either one warp
// (the batched path: thousands of shots in flight, the 32 lanes of a warp
// working on one shot) or one whole thread block of NW warps (large windows:
// every step below spread over all of the block's threads, for the latency of
// a single window).
//   1. defect compaction: the shot's syndrome bitmap is read with 16-byte
//      vector loads and compacted by a warp prefix sum (input D of the paper's
//      "Decoding task"; Alg. 1 input).
//   2. flooder: every detection event s owns an explored ball {x : dist(s,x) <=
//      R_s} with exact graph distances (hash table keyed by (vertex, event)),
//      explored once its region starts growing and kept at R_s >= Rad(s) + L
//      (L above the largest weight).  A ball is grown band by band (band >=
//      largest weight) by team-parallel label-correcting relaxation from the
//      previous band; each new entry is checked against the other events'
//      balls holding the same vertex, and against events sitting on it, which
//      records the exact distance of every pair of events whose balls touch.
//      The graph-fill region of s (SI S1) is the ball of radius Rad(s) <= R_s,
//      so two regions are found touching exactly when their pair distance
//      equals Rad(a) + Rad(b) (ARRIVE = a band extension, COLLIDE = a tight
//      pair, boundary COLLIDE = Rad(s) reaching the nearest boundary, IMPLODE =
//      an inner blossom's dual reaching 0).
//   3. Algorithm 1, level 1: each event's neighbourhood within b_1 (paths of
//      one or two edges when three smallest weights exceed b_1, else a bounded
//      search) gives every pair within b_1 and every boundary contact; min-label
//      components, the diameter <= d_1 test and the parity condition decide the
//      level-1 processing clusters.
//   4. Algorithm 2: level-1 clusters are solved independently (closed form for
//      the isolated pair and boundary singleton, the event loop otherwise), then
//      every remaining event runs from t = 0 with the stopped level-1
//      configurations present as frozen regions (hierarchical execution rule).
//      Global mode runs every event in one execution instead.
//   5. Tracing: blossoms are expanded into matched event pairs and boundary
//      matches; the weight is the sum of the tight pair / boundary distances and
//      the observable mask the XOR of the canonical paths' masks.  The
//      sliding-window instantiations (batch_kernel<true, *>) also walk every
//      path and commit the edges that touch the window's commit region.
//
// Simultaneous events are applied in the canonical order (t, kind, lo, hi) with
// kind EXTEND < IMPLODE < COLLIDE < BOUNDARY and lo, hi the ranks of the events
// in the sorted defect list, which makes the result independent of execution
// order, of the team size and equal to global sparse blossom (Theorem 1).
//
// Every loop is bounded: the event budget, hash probe lengths and list
// capacities end a shot with a status code instead of spinning.  In a team of
// several warps every decision that steers control flow around a team barrier
// is taken from a team reduction or broadcast, or from shot state that no
// thread writes between the barrier before the read and the barrier after it,
// so all threads of a team always take the same path.
//
// The rarely taken matcher steps (augment, blossom, shatter), the tracing and
// the level-1 neighbourhood searches are kept out of line (__noinline__): the
// event loop and the flooder stay inlined, and the kernel's hot code stays
// small enough for the instruction cache (each choice measured on the full
// batch; inlining the flooder or moving it out of line are both slower).

#include <algorithm>
#include <climits>
#include <cstdint>

#include "qec_internal.h"

#define WS 32   // lanes per warp
#ifndef QEC_HT_FACTOR
#define QEC_HT_FACTOR 64   // explored-table slots per detection event (rounded up to a power of two)
#endif
#ifndef QEC_MIN_BLOCKS
#define QEC_MIN_BLOCKS 6   // 128-thread blocks per SM the register budget must allow
#endif

namespace qec {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long EMPTY64 = ~0ull;
constexpr int INF32 = INT_MAX;

enum { EV_EXTEND = 0, EV_IMPLODE = 1, EV_COLLIDE = 2, EV_BOUNDARY = 3 };
constexpr int ID_BITS = 18;
constexpr int ID_MAX = (1 << ID_BITS) - 1;
constexpr long long T_MAX = (1LL << 26) - 1;

enum { MATE_NONE = -1, MATE_BOUNDARY = -2 };

// slab counters (C_R0 .. C_NEXT: work-list counters of multi-warp teams)
enum { C_ECOUNT = 0, C_WL = 1, C_NPAIRS = 2, C_CCOUNT = 3, C_NFREE = 4, C_ERR = 5, C_FRESH = 6, C_NHI = 7,
       C_TL = 8, C_CHANGED = 9, C_TNP = 10, C_TNX = 11, C_R0 = 12, C_NEXT = 15, C_TOTAL = 16 };
enum { ERR_CAP = 1, ERR_INTERNAL = 2 };

__device__ __forceinline__ unsigned long long ev_key(long long t, int kind, int lo, int hi) {
    t = t < T_MAX ? t : T_MAX;
    return ((unsigned long long)t << 38) | ((unsigned long long)kind << 36) |
           ((unsigned long long)lo << 18) | (unsigned long long)hi;
}

// Loads of per-shot state written by other threads of this team (plain stores
// or atomics): relaxed at CTA scope, so they may hit L1 and still observe every
// write ordered before them by the team's barriers.
__device__ __forceinline__ int ldr(const int *p) {
    int v;
    asm volatile("ld.relaxed.cta.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ldr(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.cta.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// One explored entry: key (vertex << 32 | source) and exact distance in one
// 16-byte slot, read by a single vector load.
struct __align__(16) HEnt {
    unsigned long long key;
    int val;
    int pad;
};
__device__ __forceinline__ void ld_ent(const HEnt *p, unsigned long long &k, int &v) {
    unsigned long long a, b;
    asm volatile("ld.relaxed.cta.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
    k = a;
    v = (int)(unsigned)(b & 0xffffffffu);
}
// Claim an empty entry (all 16 bytes ones) for (key, d) with one 16-byte
// compare-and-swap; returns true on success, else the key found there.
__device__ __forceinline__ bool claim_ent(HEnt *p, unsigned long long key, int d, unsigned long long &found) {
    const unsigned long long ek = ~0ull, ev = ~0ull;   // an empty entry is all ones
    const unsigned long long nv = (unsigned long long)(unsigned)d;
    unsigned long long ok, ov;
    asm volatile("{\n\t.reg .b128 cmp, swp, old;\n\t"
                 "mov.b128 cmp, {%2, %3};\n\t"
                 "mov.b128 swp, {%4, %5};\n\t"
                 "atom.relaxed.cta.global.cas.b128 old, [%6], cmp, swp;\n\t"
                 "mov.b128 {%0, %1}, old;\n\t}"
                 : "=l"(ok), "=l"(ov) : "l"(ek), "l"(ev), "l"(key), "l"(nv), "l"(p) : "memory");
    found = ok;
    return ok == ek && ov == ev;
}

// Claim an empty pair entry for (key, d) recording pair record idx in the
// entry's upper word; returns true on success, else the entry found there
// (key, value | record << 32).
__device__ __forceinline__ bool claim_pair(HEnt *p, unsigned long long key, int d, int idx,
                                           unsigned long long &fk, unsigned long long &fv) {
    const unsigned long long ek = ~0ull, ev = ~0ull;
    const unsigned long long nv = ((unsigned long long)(unsigned)idx << 32) | (unsigned)d;
    unsigned long long ok, ov;
    asm volatile("{\n\t.reg .b128 cmp, swp, old;\n\t"
                 "mov.b128 cmp, {%2, %3};\n\t"
                 "mov.b128 swp, {%4, %5};\n\t"
                 "atom.relaxed.cta.global.cas.b128 old, [%6], cmp, swp;\n\t"
                 "mov.b128 {%0, %1}, old;\n\t}"
                 : "=l"(ok), "=l"(ov) : "l"(ek), "l"(ev), "l"(key), "l"(nv), "l"(p) : "memory");
    fk = ok;
    fv = ov;
    return ok == ek && ov == ev;
}

// Warp-aggregated atomicAdd(ctr, 1) over the currently active lanes.
__device__ __forceinline__ int agg_inc(int *ctr, int lane) {
    const unsigned m = __activemask();
    const int leader = __ffs(m) - 1;
    const int rank = __popc(m & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(ctr, __popc(m));
    base = __shfl_sync(m, base, leader);
    return base + rank;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
#pragma unroll
    for (int o = WS / 2; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(FULL, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// The same with the 32-bit reduction unit: the smallest high word, then the
// smallest low word among the lanes holding it (faster in a block-wide team,
// measured slower in the one-warp path).
__device__ __forceinline__ unsigned long long warp_min64_redux(unsigned long long v) {
    const unsigned hi = (unsigned)(v >> 32);
    const unsigned mh = __reduce_min_sync(FULL, hi);
    const unsigned ml = __reduce_min_sync(FULL, hi == mh ? (unsigned)v : 0xffffffffu);
    return ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = WS / 2; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_xor64(unsigned long long v) {
#pragma unroll
    for (int o = WS / 2; o; o >>= 1) v ^= __shfl_xor_sync(FULL, v, o);
    return v;
}

// ------------------------------------------------------------------ teams --

// Shared scratch of a multi-warp team: one slot per warp for reductions, in
// two alternating buffers (every team operation ends with one barrier, so a
// buffer is reused only after every thread has read it).  Functions kept out
// of line take their Team by value and end with a barrier after their last
// team operation, so the caller may go on with its own buffer parity.
struct __align__(16) TSlot {
    unsigned long long u;
    int a, b;
};
struct TeamShared {
    TSlot s[2][32];
};

// Per-thread identity of a team member: a one-warp team needs only the lane
// (its thread index is the lane, its warp 0, and it has no shared scratch).
template <int NW>
struct TeamId {
    int tid_, lane, warp_, ph;
    TeamShared *sh;
    __device__ __forceinline__ int tid() const { return tid_; }
    __device__ __forceinline__ int warp() const { return warp_; }
};
template <>
struct TeamId<1> {
    int lane;
    __device__ __forceinline__ int tid() const { return lane; }
    __device__ __forceinline__ int warp() const { return 0; }
};

template <int NW>
struct Team : TeamId<NW> {
    static constexpr int NT = WS * NW;
    using TeamId<NW>::lane;
    using TeamId<NW>::tid;
    using TeamId<NW>::warp;

    __device__ __forceinline__ void sync() const {
        if constexpr (NW == 1) __syncwarp(); else __syncthreads();
    }
    // thread 0's value for every thread
    __device__ __forceinline__ int bcast(int v) {
        if constexpr (NW == 1) {
            return __shfl_sync(FULL, v, 0);
        } else {
            if (tid() == 0) this->sh->s[this->ph][0].a = v;
            __syncthreads();
            v = this->sh->s[this->ph][0].a;
            this->ph ^= 1;
            return v;
        }
    }
    __device__ __forceinline__ unsigned long long bcast64(unsigned long long v) {
        if constexpr (NW == 1) {
            return __shfl_sync(FULL, v, 0);
        } else {
            if (tid() == 0) this->sh->s[this->ph][0].u = v;
            __syncthreads();
            v = this->sh->s[this->ph][0].u;
            this->ph ^= 1;
            return v;
        }
    }
    // Cross-warp stage of a block reduction: lane 0 of every warp stores its
    // warp's value in its slot; after the barrier lane w of every warp reads
    // slot w (one 16-byte load), and each warp reduces those NW values itself.
    __device__ __forceinline__ TSlot gather(const TSlot &mine, const TSlot &identity) {
        if (lane == 0) this->sh->s[this->ph][warp()] = mine;
        __syncthreads();
        const TSlot x = lane < NW ? this->sh->s[this->ph][lane] : identity;
        this->ph ^= 1;
        return x;
    }
    __device__ __forceinline__ unsigned long long min64(unsigned long long v) {
        if constexpr (NW == 1) return warp_min64(v);
        else return warp_min64_redux(gather(TSlot{warp_min64_redux(v), 0, 0}, TSlot{EMPTY64, 0, 0}).u);
    }
    __device__ __forceinline__ long long sum64(long long v) {
        v = warp_sum64(v);
        if constexpr (NW == 1) return v;
        else return warp_sum64((long long)gather(TSlot{(unsigned long long)v, 0, 0}, TSlot{0, 0, 0}).u);
    }
    __device__ __forceinline__ unsigned long long xor64(unsigned long long v) {
        v = warp_xor64(v);
        if constexpr (NW == 1) return v;
        else return warp_xor64(gather(TSlot{v, 0, 0}, TSlot{0, 0, 0}).u);
    }
    // op: 0 = add, 1 = max, 2 = or
    template <int OP>
    __device__ __forceinline__ int warp_red32(int v) {
        if constexpr (OP == 0) return (int)__reduce_add_sync(FULL, (unsigned)v);
        else if constexpr (OP == 1) return __reduce_max_sync(FULL, v);
        else return (int)__reduce_or_sync(FULL, (unsigned)v);
    }
    template <int OP>
    __device__ __forceinline__ int red32(int v) {
        v = warp_red32<OP>(v);
        if constexpr (NW == 1) return v;
        else return warp_red32<OP>(gather(TSlot{0, v, 0}, TSlot{0, OP == 1 ? INT_MIN : 0, 0}).a);
    }
    __device__ __forceinline__ int add(int v) { return red32<0>(v); }
    __device__ __forceinline__ int maxi(int v) { return red32<1>(v); }
    __device__ __forceinline__ bool any(bool b) { return red32<2>(b ? 1 : 0) != 0; }
    // The event search's reduction in one barrier: smallest key, OR of flags,
    // smallest m (as unsigned).
    __device__ __forceinline__ void reduce_ev(unsigned long long &key, int &flags, unsigned &m) {
        if constexpr (NW == 1) key = warp_min64(key);
        else key = warp_min64_redux(key);
        flags = (int)__reduce_or_sync(FULL, (unsigned)flags);
        m = __reduce_min_sync(FULL, m);
        if constexpr (NW > 1) {
            const TSlot x = gather(TSlot{key, flags, (int)m}, TSlot{EMPTY64, 0, -1});
            key = warp_min64_redux(x.u);
            flags = (int)__reduce_or_sync(FULL, (unsigned)x.a);
            m = __reduce_min_sync(FULL, (unsigned)x.b);
        }
    }
    // Exclusive prefix sum of v over the team's threads in tid order; `total`
    // receives the sum over all threads.
    __device__ __forceinline__ int excl_scan(int v, int &total) {
        int incl = v;
#pragma unroll
        for (int o = 1; o < WS; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int wtot = __shfl_sync(FULL, incl, WS - 1);
        if constexpr (NW == 1) {
            total = wtot;
            return incl - v;
        } else {
            // lane w holds warp w's total: the warp's offset and the block total
            const int x = gather(TSlot{0, wtot, 0}, TSlot{0, 0, 0}).a;
            const int off = (int)__reduce_add_sync(FULL, (unsigned)(lane < warp() ? x : 0));
            total = (int)__reduce_add_sync(FULL, (unsigned)x);
            return off + incl - v;
        }
    }
};

// Per-source state read together by the event search, the dual update and
// the EXTEND scan: one 16-byte record (a single vector load).
//   stop: top-level matcher node containing the source; srad: Rad(s);
//   sR: explored radius (-1: never explored); inplay: part of the current run;
//   sexh: ball exhausted (no vertex left to explore).
struct __align__(16) SRec {
    int stop, srad, sR;
    unsigned char inplay, sexh, pad0, pad1;
};
__device__ __forceinline__ int4 ld_src(const SRec *p) { return *reinterpret_cast<const int4 *>(p); }
__device__ __forceinline__ int rec_inplay(const int4 &r) { return r.w & 0xff; }
__device__ __forceinline__ int rec_sexh(const int4 &r) { return (r.w >> 8) & 0xff; }

// Matcher node state read together by the node scans (dual update,
// implosions, fix-ups): y = the node's own dual, bpar = parent blossom (-1:
// top level), label = +1 outer / -1 inner / 0 not in a tree, alive.
struct __align__(16) NRec {
    int y, bpar, label, alive;
};
__device__ __forceinline__ int4 ld_nd(const NRec *p) { return *reinterpret_cast<const int4 *>(p); }

// A pair of events whose balls met, as a block-wide team keeps it: ranks
// lo < hi, exact distance (equal to the hash entry's value after every
// barrier), hash slot.  All ones (lo = -1) is an unused record: a record
// reserved by an insert that lost the race for its slot to the same pair
// stays so.  A one-warp team lists the pairs' hash slots instead (plist).
struct __align__(16) PRec {
    int lo, hi;
    unsigned val;
    int slot;
};
__device__ __forceinline__ int4 ld_pr(const PRec *p) { return *reinterpret_cast<const int4 *>(p); }

struct Slab {
    // per detection event (source)
    SRec *src;
    int *svtx, *sbeg, *scnt, *comp, *cst0, *cst1, *cst2;
    unsigned long long *sbnd;
    // explored entries (open addressing, keyed by vertex and source); `ent`
    // holds the table slots of every source's bands (band lists)
    HEnt *ht;
    int *ent;
    unsigned long long *wl0, *wl1, *tl;   // work lists (table slots) / new entries (slot << 32 | position)
    int *xsrc, *xR, *xcnt, *xcur;         // sources being extended, target radii, band counts
    int *xidx;                            // position of a source in xsrc during an extension
    int *wcum;                            // detection events in syndrome words before word w
    // pairs: key (lo << 32 | hi), value distance; one-warp teams list the
    // used slots (plist), block-wide teams keep pair records (pr, carved
    // last) whose index the hash entry's upper word holds
    HEnt *pt;
    int *plist;
    PRec *pr;
    // matcher nodes (leaf s = node s, blossoms above K)
    NRec *nd;
    int *tpar, *tps, *tpo, *mate, *ms, *mo, *nroot, *minleaf, *cbeg, *clen, *freel, *tmpa, *tmpb, *stk;
    int *cnode, *cs, *co;
    int *ctr;
};

template <typename T>
__host__ __device__ inline T *bump(char *&p, long long n) {
    uintptr_t q = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    T *r = reinterpret_cast<T *>(q);
    p = reinterpret_cast<char *>(q + sizeof(T) * (size_t)n);
    return r;
}

__host__ __device__ inline long long carve(char *base, const SlabCaps &c, Slab &S) {
    char *p = base;
    S.src = bump<SRec>(p, c.kc);
    S.svtx = bump<int>(p, c.kc); S.sbeg = bump<int>(p, c.kc); S.scnt = bump<int>(p, c.kc);
    S.comp = bump<int>(p, c.kc);
    S.cst0 = bump<int>(p, c.kc); S.cst1 = bump<int>(p, c.kc); S.cst2 = bump<int>(p, c.kc);
    S.sbnd = bump<unsigned long long>(p, c.kc);
    S.ht = bump<HEnt>(p, c.hc);
    S.ent = bump<int>(p, c.ec);
    S.wl0 = bump<unsigned long long>(p, c.wc); S.wl1 = bump<unsigned long long>(p, c.wc);
    S.tl = bump<unsigned long long>(p, c.ec);
    S.xsrc = bump<int>(p, c.kc); S.xR = bump<int>(p, c.kc); S.xcnt = bump<int>(p, c.kc); S.xcur = bump<int>(p, c.kc);
    S.xidx = bump<int>(p, c.kc);
    S.wcum = bump<int>(p, c.wcap);
    S.pt = bump<HEnt>(p, c.phc); S.plist = bump<int>(p, c.phc);
    S.nd = bump<NRec>(p, c.nc);
    S.tpar = bump<int>(p, c.nc); S.tps = bump<int>(p, c.nc); S.tpo = bump<int>(p, c.nc);
    S.mate = bump<int>(p, c.nc); S.ms = bump<int>(p, c.nc); S.mo = bump<int>(p, c.nc);
    S.nroot = bump<int>(p, c.nc); S.minleaf = bump<int>(p, c.nc); S.cbeg = bump<int>(p, c.nc);
    S.clen = bump<int>(p, c.nc); S.freel = bump<int>(p, c.nc);
    S.tmpa = bump<int>(p, 2 * c.nc + 64); S.tmpb = bump<int>(p, 2 * c.nc + 64);
    S.stk = bump<int>(p, 4 * c.nc + 64);
    S.cnode = bump<int>(p, c.cc); S.cs = bump<int>(p, c.cc); S.co = bump<int>(p, c.cc);
    S.ctr = bump<int>(p, C_TOTAL);
    S.pr = bump<PRec>(p, (c.phc >> 1) + 1);   // last: the one-warp layout above is unchanged
    return (long long)(p - base) + 16;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Shot {
    unsigned long long deadline;   // globaltimer value after which the shot gives up (0 = none)
    DGraph g;
    int K;            // detection events
    unsigned hmask;   // explored-entry hash mask
    unsigned pmask;   // pair hash mask
    int ec, wc, nc, cc;
    int band;
    int L;                 // lookahead: explored radius >= Rad + L for every growing region
    const unsigned *row;   // the shot's syndrome row (defect test)
    long long t;
    long long events;
    long long max_events;
    // parallel-event-count bookkeeping of the current run (Methods, "Numerical
    // evaluation"): matcher events applied, those at times <= tcut, the time of
    // the last one, and flooder band extensions
    int nm, ncut, tcut, tlast, nx;
};

// Home slots: the high bits of a multiplicative (Fibonacci) hash, so that
// nearby vertices spread over the whole table; mask + 1 is a power of two.
__device__ __forceinline__ unsigned hslot(int v, unsigned mask) {
    return ((unsigned)v * 2654435761u) >> (32 - __popc(mask));
}

__device__ __forceinline__ unsigned pslot(int lo, int hi, unsigned mask) {
    return (((unsigned)lo * 2654435761u + (unsigned)hi) * 2246822519u) >> (32 - __popc(mask));
}

__device__ __forceinline__ void set_err(const Slab &S, int bit) { atomicOr(&S.ctr[C_ERR], bit); }

// exact distance of (v, s) if explored, else INF32
__device__ int ht_get(const Slab &S, const Shot &C, int v, int s) {
    const unsigned long long key = ((unsigned long long)(unsigned)v << 32) | (unsigned)s;
    unsigned i = hslot(v, C.hmask);
    for (unsigned n = 0; n <= C.hmask; n++) {
        unsigned long long k;
        int v;
        ld_ent(&S.ht[i], k, v);
        if (k == key) return v;
        if (k == EMPTY64) return INF32;
        i = (i + 1) & C.hmask;
    }
    return INF32;
}

// insert-or-decrease; returns 1 inserted, 2 decreased, 0 unchanged, -1 table
// full; `slot` receives the entry's table slot
__device__ int ht_upsert(const Slab &S, const Shot &C, int v, int s, int d, unsigned &slot) {
    const unsigned long long key = ((unsigned long long)(unsigned)v << 32) | (unsigned)s;
    unsigned i = hslot(v, C.hmask);
    for (unsigned n = 0; n <= C.hmask; n++) {
        unsigned long long k;
        int v;
        ld_ent(&S.ht[i], k, v);
        if (k == EMPTY64) {
            if (claim_ent(&S.ht[i], key, d, k)) {
                slot = i;
                return 1;
            }
            v = INF32;
        }
        if (k == key) {
            slot = i;
            if (d >= v) return 0;   // values only decrease: nothing to do
            int old = atomicMin(&S.ht[i].val, d);
            return d < old ? 2 : 0;
        }
        i = (i + 1) & C.hmask;
    }
    set_err(S, ERR_CAP);
    return -1;
}

// Insert-or-decrease the pair (a, b) with distance d.  REC (block-wide
// teams): a new pair reserves the next pair record before claiming its slot,
// and every value written to the hash entry is also applied to the record by
// the thread that wrote it, so both hold the minimum after the next barrier.
// Otherwise the claimed slot is appended to the pair list.
template <bool REC>
__device__ void pair_upsert(const Slab &S, const Shot &C, int a, int b, int d) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    const unsigned long long key = ((unsigned long long)(unsigned)lo << 32) | (unsigned)hi;
    unsigned i = pslot(lo, hi, C.pmask);
    if constexpr (REC) {
        int idx = -1;
        for (unsigned n = 0; n <= C.pmask; n++) {
            unsigned long long k, w;
            asm volatile("ld.relaxed.cta.v2.b64 {%0, %1}, [%2];" : "=l"(k), "=l"(w) : "l"(&S.pt[i]) : "memory");
            if (k == EMPTY64) {
                if (idx < 0) {
                    idx = atomicAdd(&S.ctr[C_NPAIRS], 1);
                    if ((unsigned)idx * 2u > C.pmask) { set_err(S, ERR_CAP); return; }
                }
                if (claim_pair(&S.pt[i], key, d, idx, k, w)) {
                    S.pr[idx].lo = lo; S.pr[idx].hi = hi; S.pr[idx].slot = (int)i;
                    atomicMin(&S.pr[idx].val, (unsigned)d);
                    return;
                }
            }
            if (k == key) {
                const int v = (int)(unsigned)(w & 0xffffffffu), j = (int)(w >> 32);
                if (d < v) {
                    atomicMin(&S.pt[i].val, d);
                    atomicMin(&S.pr[j].val, (unsigned)d);
                }
                return;   // a reserved record stays unused
            }
            i = (i + 1) & C.pmask;
        }
    } else {
        for (unsigned n = 0; n <= C.pmask; n++) {
            unsigned long long k;
            int v;
            ld_ent(&S.pt[i], k, v);
            if (k == EMPTY64) {
                if (claim_ent(&S.pt[i], key, d, k)) {
                    int idx = atomicAdd(&S.ctr[C_NPAIRS], 1);
                    if ((unsigned)idx * 2u > C.pmask) set_err(S, ERR_CAP);
                    else S.plist[idx] = (int)i;
                    return;
                }
                v = INF32;
            }
            if (k == key) {
                if (d < v) atomicMin(&S.pt[i].val, d);
                return;
            }
            i = (i + 1) & C.pmask;
        }
    }
    set_err(S, ERR_CAP);
}

__device__ int pair_get(const Slab &S, const Shot &C, int a, int b) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    const unsigned long long key = ((unsigned long long)(unsigned)lo << 32) | (unsigned)hi;
    unsigned i = pslot(lo, hi, C.pmask);
    for (unsigned n = 0; n <= C.pmask; n++) {
        unsigned long long k;
        int v;
        ld_ent(&S.pt[i], k, v);
        if (k == key) return v;
        if (k == EMPTY64) return INF32;
        i = (i + 1) & C.pmask;
    }
    return INF32;
}

// The i-th pair found (ranks a < b, distance pv); false for an unused record.
template <int NW>
__device__ __forceinline__ bool pair_at(const Slab &S, int i, int &a, int &b, int &pv) {
    if constexpr (NW == 1) {
        unsigned long long k;
        ld_ent(&S.pt[S.plist[i]], k, pv);
        a = (int)(k >> 32); b = (int)(unsigned)(k & 0xffffffffu);
        return true;
    } else {
        const int4 pq = ld_pr(&S.pr[i]);
        a = pq.x; b = pq.y; pv = pq.z;
        return a >= 0;
    }
}

struct SlotV {
    int nbr;   // neighbour detector, -1 for the boundary
    int w;     // internal weight
    int eid;   // merged edge id (boundary slots only; -1 otherwise)
};

__device__ __forceinline__ SlotV load_slot(const DGraph &g, int j) {
    const int2 v = __ldg(reinterpret_cast<const int2 *>(g.slot) + j);
    SlotV s;
    s.w = v.y;
    if (v.x < 0) { s.nbr = -1; s.eid = -1 - v.x; }
    else { s.nbr = v.x; s.eid = -1; }
    return s;
}

__device__ __forceinline__ bool is_defect(const Shot &C, int v) {
    return (__ldg(C.row + (v >> 5)) >> (v & 31)) & 1u;
}

// Rank of detection event vertex v in the sorted event list (v must be an
// event): events in earlier words plus set bits below v in its own word.
__device__ __forceinline__ int rank_of(const Slab &S, const Shot &C, int v) {
    const unsigned w = __ldg(C.row + (v >> 5));
    return S.wcum[v >> 5] + __popc(w & ((1u << (v & 31)) - 1u));
}

__device__ __forceinline__ void bnd_update(const Slab &S, int s, int d, int eid) {
    unsigned long long v = ((unsigned long long)(unsigned)d << 32) | (unsigned)eid;
    atomicMin(&S.sbnd[s], v);
}

// Grow the explored balls of the sources xsrc[0 .. nx) from radius sR[s] to
// xR[i] (xR[i] - sR[s] >= largest weight), all at once: the previous band of
// each source is the frontier, label-correcting relaxation runs on work lists
// of table slots (a slot's key names the vertex and source, its value the
// current distance) until no distance changes, every new entry is checked for
// contacts with the other sources' balls, and each source's new band is stored
// contiguously in `ent` as its next frontier.  Every thread of the team calls
// with the same nx.
template <int NW>
__device__ void extend_many(const Slab &S, const Shot &C, int nx, Team<NW> &T) {
    const DGraph &g = C.g;
    if (nx <= 0) return;
    const int lane = T.lane;
    T.sync();
    if (T.tid() == 0) {
        S.ctr[C_TL] = 0; S.ctr[C_WL] = 0; S.ctr[C_FRESH] = 0;
        if constexpr (NW > 1) { S.ctr[C_R0] = 0; S.ctr[C_R0 + 1] = 0; }
    }
    for (int i = T.tid(); i < nx; i += T.NT) { S.xcnt[i] = 0; S.xidx[S.xsrc[i]] = i; }
    T.sync();
    unsigned *F = reinterpret_cast<unsigned *>(S.wl0), *Wn = reinterpret_cast<unsigned *>(S.wl1);
    // A source never explored whose target radius is below three smallest
    // weights has a first ball made of paths of at most two edges: it is
    // enumerated directly below (listed in xcur).  Initial frontier of the
    // others: the previous band of every listed source; a source never
    // explored so far starts from its own vertex at distance 0.
    const int r3 = 3 * g.wmin;
    for (int i = T.tid(); i < nx; i += T.NT) {
        const int s = S.xsrc[i];
        if (S.src[s].sR < 0 && S.xR[i] < r3) {
            S.xcur[atomicAdd(&S.ctr[C_FRESH], 1)] = i;
            continue;
        }
        if (S.src[s].sR < 0) {
            unsigned hs;
            const int r = ht_upsert(S, C, S.svtx[s], s, 0, hs);
            if (r < 0) continue;
            if (r == 1) {
                const int e = atomicAdd(&S.ctr[C_TL], 1);
                if (e < C.ec) S.tl[e] = ((unsigned long long)hs << 32) | (unsigned)i; else set_err(S, ERR_CAP);
            }
            const int w = atomicAdd(&S.ctr[C_WL], 1);
            if (w < C.wc) F[w] = hs; else set_err(S, ERR_CAP);
            continue;
        }
        const int fb = S.sbeg[s], fc = S.scnt[s];
        const int base = atomicAdd(&S.ctr[C_WL], fc);
        for (int k = 0; k < fc; k++) {
            if (base + k < C.wc) F[base + k] = (unsigned)S.ent[fb + k];
            else set_err(S, ERR_CAP);
        }
    }
    T.sync();
    int nf = min(ldr(&S.ctr[C_WL]), C.wc);
    // a one-warp team keeps the list counters in registers (warp-uniform) and
    // places each round's appends by ballot; several warps reserve their
    // appends with one atomic per warp and round on counters that rotate over
    // three slots (a slot is cleared two rounds before its next use)
    int ntl = ldr(&S.ctr[C_TL]);
    const unsigned lt = (1u << lane) - 1u;
    // new explored entry (table slot hs) of list position xi: one slot in `tl`
    // per inserted entry, placed by ballot (one warp) or by one atomic per warp
    auto append_tl = [&](bool ins, unsigned hs, int xi) {
        const unsigned mt = __ballot_sync(FULL, ins);
        int bt;
        if constexpr (NW == 1) {
            bt = ntl;
            ntl += __popc(mt);
        } else {
            bt = 0;
            if (lane == 0 && mt) bt = atomicAdd(&S.ctr[C_TL], __popc(mt));
            bt = __shfl_sync(FULL, bt, 0);
        }
        if (ins) {
            const int e = bt + __popc(mt & lt);
            if (e < C.ec) S.tl[e] = ((unsigned long long)hs << 32) | (unsigned)xi; else set_err(S, ERR_CAP);
        }
    };
    {
        // first balls by enumeration: every vertex within radius R of the
        // source is reached by a path of one or two edges, so the minimum over
        // those paths is its exact distance; boundary candidates through the
        // source and its neighbours (the band's farther vertices are the next
        // extension's frontier, which adds theirs before a region can get
        // there).  One lane per (source, adjacency slot), as in level1_2hop.
        const int nfr = ldr(&S.ctr[C_FRESH]);
        for (int base = T.warp() * WS; base < nfr; base += T.NT) {
            const int idx = base + lane;
            int src = -1, r0 = 0, deg = 0, xi = 0, s = 0, R = -1;
            bool ins = false;
            unsigned hs = 0;
            if (idx < nfr) {
                xi = S.xcur[idx];
                s = S.xsrc[xi];
                R = S.xR[xi];
                src = S.svtx[s];
                r0 = __ldg(g.row + src);
                deg = __ldg(g.row + src + 1) - r0;
                ins = ht_upsert(S, C, src, s, 0, hs) == 1;
            }
            append_tl(ins, hs, xi);
            int incl = deg;
            for (int o = 1; o < WS; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(FULL, incl, WS - 1);
            const int excl = incl - deg;
            for (int t0 = 0; t0 < total; t0 += WS) {
                const int t = t0 + lane;
                int ow = 0;
                for (int step = WS / 2; step > 0; step >>= 1) {
                    const int e = __shfl_sync(FULL, excl, ow + step);
                    if (e <= t) ow += step;
                }
                const int osrc = __shfl_sync(FULL, src, ow);
                const int oj = __shfl_sync(FULL, r0 - excl, ow) + t;
                const int os = __shfl_sync(FULL, s, ow);
                const int oR = __shfl_sync(FULL, R, ow);
                const int oxi = __shfl_sync(FULL, xi, ow);
                int an = -1, aw = 0;
                bool ins1 = false;
                unsigned h1 = 0;
                if (t < total) {
                    const SlotV a = load_slot(g, oj);
                    aw = a.w;
                    if (a.nbr < 0) bnd_update(S, os, a.w, a.eid);
                    else if (a.w <= oR) {
                        an = a.nbr;
                        ins1 = ht_upsert(S, C, an, os, a.w, h1) == 1;
                    }
                }
                append_tl(ins1, h1, oxi);
                // second edges from the neighbour, one lane each
                const int q0 = an >= 0 ? __ldg(g.row + an) : 0, q1 = an >= 0 ? __ldg(g.row + an + 1) : 0;
                const int nq = __reduce_max_sync(FULL, (unsigned)(q1 - q0));
                for (int k = 0; k < nq; k++) {
                    bool ins2 = false;
                    unsigned h2 = 0;
                    if (k < q1 - q0) {
                        const SlotV b = load_slot(g, q0 + k);
                        const int nd = aw + b.w;
                        if (b.nbr < 0) bnd_update(S, os, nd, b.eid);
                        else if (nd <= oR && b.nbr != osrc) ins2 = ht_upsert(S, C, b.nbr, os, nd, h2) == 1;
                    }
                    append_tl(ins2, h2, oxi);
                }
            }
        }
    }
    for (int iter = 0;; iter++) {
        if (iter >= 4096) { if (T.tid() == 0) set_err(S, ERR_INTERNAL); break; }
        int nwl = 0;
        int *const wctr = &S.ctr[C_R0 + iter % 3];
        if constexpr (NW > 1) {
            if (T.tid() == 0) S.ctr[C_R0 + (iter + 1) % 3] = 0;
        }
        // one lane per (work item, adjacency slot): items are taken 32 at a
        // time per warp, their slots numbered by a warp prefix sum of the
        // degrees, and slot t goes to lane t mod 32 (its item found by binary
        // search)
        for (int base = T.warp() * WS; base < nf; base += T.NT) {
            const int i = base + lane;
            unsigned long long key = 0;
            int dx = 0, Rn = -1, r0 = 0, deg = 0, xi = 0;
            if (i < nf) {
                const unsigned hx = F[i];
                ld_ent(&S.ht[hx], key, dx);
                const int x = (int)(key >> 32);
                xi = S.xidx[(int)(unsigned)(key & 0xffffffffu)];
                Rn = S.xR[xi];
                r0 = __ldg(g.row + x);
                deg = __ldg(g.row + x + 1) - r0;
            }
            int incl = deg;
            for (int o = 1; o < WS; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(FULL, incl, WS - 1);
            const int excl = incl - deg;
            for (int t0 = 0; t0 < total; t0 += WS) {
                const int t = t0 + lane;
                // owner: the last lane whose first slot number is <= t
                int ow = 0;
                for (int step = WS / 2; step > 0; step >>= 1) {
                    const int e = __shfl_sync(FULL, excl, ow + step);
                    if (e <= t) ow += step;
                }
                const unsigned long long okey = __shfl_sync(FULL, key, ow);
                const int odx = __shfl_sync(FULL, dx, ow);
                const int oRn = __shfl_sync(FULL, Rn, ow);
                const int oj = __shfl_sync(FULL, r0 - excl, ow) + t;
                const int oxi = __shfl_sync(FULL, xi, ow);
                int r = 0;
                unsigned hs = 0;
                if (t < total) {
                    const int s = (int)(unsigned)(okey & 0xffffffffu);
                    const SlotV sl = load_slot(g, oj);
                    const int nd = odx + sl.w;
                    if (sl.nbr < 0) bnd_update(S, s, nd, sl.eid);
                    else if (nd <= oRn) r = ht_upsert(S, C, sl.nbr, s, nd, hs);
                }
                const unsigned mt = __ballot_sync(FULL, r == 1);
                const unsigned mw = __ballot_sync(FULL, r >= 1);
                int bt, bw;
                if constexpr (NW == 1) {
                    bt = ntl; bw = nwl;
                    ntl += __popc(mt);
                    nwl += __popc(mw);
                } else {
                    bt = 0; bw = 0;
                    if (lane == 0) {
                        if (mt) bt = atomicAdd(&S.ctr[C_TL], __popc(mt));
                        if (mw) bw = atomicAdd(wctr, __popc(mw));
                    }
                    bt = __shfl_sync(FULL, bt, 0);
                    bw = __shfl_sync(FULL, bw, 0);
                }
                if (r == 1) {
                    const int e = bt + __popc(mt & lt);
                    if (e < C.ec) S.tl[e] = ((unsigned long long)hs << 32) | (unsigned)oxi; else set_err(S, ERR_CAP);
                }
                if (r >= 1) {
                    const int w = bw + __popc(mw & lt);
                    if (w < C.wc) Wn[w] = hs; else set_err(S, ERR_CAP);
                }
            }
        }
        T.sync();
        bool stop;
        if constexpr (NW == 1) {
            const int err = ldr(&S.ctr[C_ERR]);
            stop = nwl == 0 || err;
        } else {
            // this round's counter is written by no thread until two rounds
            // on, so every thread reads the same value: a uniform decision
            // without a reduction (a capacity error ends the rounds once no
            // insertion succeeds; the caller reads the error word)
            nwl = ldr(wctr);
            stop = nwl == 0;
        }
        if (stop) break;
        nf = min(nwl, C.wc);
        unsigned *t = F; F = Wn; Wn = t;
    }
    if constexpr (NW == 1) {
        if (lane == 0) S.ctr[C_TL] = ntl;
    }
    T.sync();
    const unsigned long long ne = T.bcast64(((unsigned long long)(unsigned)min(ldr(&S.ctr[C_TL]), C.ec) << 32) |
                                            (unsigned)ldr(&S.ctr[C_ECOUNT]));
    const int nt = (int)(unsigned)(ne >> 32);
    const int e0 = (int)(unsigned)(ne & 0xffffffffu);
    // explored-entry table at most half full, list room left
    if (e0 + nt > C.ec || (unsigned)(e0 + nt) * 2u > C.hmask) {
        if (T.tid() == 0) set_err(S, ERR_CAP);
        T.sync();
        return;
    }
    // bands made contiguous per source (counting sort of the new entries)
    for (int i = T.tid(); i < nt; i += T.NT) atomicAdd(&S.xcnt[(int)(unsigned)(S.tl[i] & 0xffffffffu)], 1);
    T.sync();
    if constexpr (NW == 1) {
        // band starts in list order, by lane 0 (a warp extends only a few
        // sources at a time; measured faster than a warp-wide scan)
        if (lane == 0) {
            int acc = e0;
            for (int i = 0; i < nx; i++) {
                const int s = S.xsrc[i];
                const int c = S.xcnt[i];
                S.xcur[i] = acc;
                S.sbeg[s] = acc;
                S.scnt[s] = c;
                S.src[s].sR = S.xR[i];
                if (c == 0) S.src[s].sexh = 1;
                acc += c;
            }
            S.ctr[C_ECOUNT] = acc;
        }
    } else {
        // band starts: exclusive prefix sum of the counts in list order, each
        // thread one contiguous chunk of the list
        const int per = (nx + T.NT - 1) / T.NT;
        const int i0 = min(nx, T.tid() * per), i1 = min(nx, i0 + per);
        int loc = 0;
        for (int i = i0; i < i1; i++) loc += S.xcnt[i];
        int total = 0;
        int acc = e0 + T.excl_scan(loc, total);
        for (int i = i0; i < i1; i++) {
            const int s = S.xsrc[i];
            const int c = S.xcnt[i];
            S.xcur[i] = acc;
            S.sbeg[s] = acc;
            S.scnt[s] = c;
            S.src[s].sR = S.xR[i];
            if (c == 0) S.src[s].sexh = 1;
            acc += c;
        }
        if (T.tid() == 0) {
            S.ctr[C_ECOUNT] = e0 + total;
            S.ctr[C_NEXT] = 0;
        }
    }
    T.sync();
    for (int i = T.tid(); i < nt; i += T.NT) {
        const unsigned long long it = S.tl[i];
        const int pos = atomicAdd(&S.xcur[(int)(unsigned)(it & 0xffffffffu)], 1);
        S.ent[pos] = (int)(it >> 32);
    }
    T.sync();
    // contacts of every new entry y of source s: other explored balls holding y
    // (same vertex), and y being another detection event's own vertex (reach).
    // With explored radius >= Rad + L for every growing region (L >= largest
    // weight, >= the radius of any never-explored frozen region) these find every
    // pair of regions at the instant they become tight: on a shortest path
    // between them, the first vertex at distance >= Rad(a) from a lies in b's
    // region and within Rad(a) + largest weight of a.
    // Each lane walks the probe chain of one entry, one probe per round; a lane
    // whose walk has ended takes the next unwalked entry, so the lanes stay busy
    // however the chain lengths vary (a warp of a larger team claims entries
    // from a shared counter).
    {
        int cur = -1, yv = 0, s = 0, dy = 0;
        unsigned pos = 0, nprobe = 0;
        int next = 0;
        for (long long round = 0; round < (long long)nt * (C.hmask + 2) + 1; round++) {
            const unsigned idle = __ballot_sync(FULL, cur < 0);
            int kb;
            if constexpr (NW == 1) {
                kb = next;
                next += __popc(idle);
            } else {
                kb = 0;
                if (lane == 0 && idle) kb = atomicAdd(&S.ctr[C_NEXT], __popc(idle));
                kb = __shfl_sync(FULL, kb, 0);
            }
            if (cur < 0) {
                const int k = kb + __popc(idle & lt);
                if (k < nt) {
                    cur = k;
                    const unsigned hy = (unsigned)(S.tl[k] >> 32);
                    unsigned long long key;
                    ld_ent(&S.ht[hy], key, dy);
                    yv = (int)(key >> 32);
                    s = (int)(unsigned)(key & 0xffffffffu);
                    pos = hslot(yv, C.hmask);
                    nprobe = 0;
                    if (yv != S.svtx[s] && is_defect(C, yv)) {
                        const int f = rank_of(S, C, yv);
                        if (f >= 0 && f != s) pair_upsert<(NW > 1)>(S, C, s, f, dy);
                    }
                }
            }
            if (!__any_sync(FULL, cur >= 0)) break;
            if (cur >= 0) {
                unsigned long long k;
                int v;
                ld_ent(&S.ht[pos], k, v);
                if (k == EMPTY64 || ++nprobe > C.hmask) {
                    cur = -1;
                } else {
                    if ((int)(k >> 32) == yv) {
                        const int s2 = (int)(unsigned)(k & 0xffffffffu);
                        if (s2 != s) pair_upsert<(NW > 1)>(S, C, s, s2, dy + v);
                    }
                    pos = (pos + 1) & C.hmask;
                }
            }
        }
    }
    T.sync();
}

// Grow one source's ball by one band.  Every thread of the team calls.
template <int NW>
__device__ void extend_one(const Slab &S, const Shot &C, int s, Team<NW> &T) {
    if (T.tid() == 0) { S.xsrc[0] = s; S.xR[0] = max(S.src[s].sR, 0) + C.band; }
    T.sync();
    extend_many(S, C, 1, T);
}

// ---------------------------------------------------------------- matcher --

// Child of blossom B that contains `leaf` (-1 if B is not an ancestor).
__device__ __forceinline__ int child_of(const Slab &S, int B, int leaf) {
    int v = leaf;
    for (int n = 0; n < 1 << 20 && v >= 0 && S.nd[v].bpar != B; n++) v = S.nd[v].bpar;
    return v;
}

// flip matches along the tree path from outer A to its root (thread 0)
__device__ void flip_to_root(const Slab &S, int A) {
    int v = A;
    for (int n = 0; n < 1 << 22 && S.tpar[v] >= 0; n++) {
        const int I = S.tpar[v];
        const int O = S.tpar[I];
        if (O < 0) { S.ctr[C_ERR] |= ERR_INTERNAL; return; }
        S.mate[I] = O; S.ms[I] = S.tps[I]; S.mo[I] = S.tpo[I];
        S.mate[O] = I; S.ms[O] = S.tpo[I]; S.mo[O] = S.tps[I];
        v = O;
    }
}

// Events (b), (f), (g).  B < 0: boundary.  Every thread of the team calls.
template <int NW>
__device__ __noinline__ void ev_augment(const Slab &S, Shot &C, int A, int a, int B, int b, Team<NW> T, int nhi) {
    int rA = 0, rB = -3;
    bool bout = false;
    // flip the matches along both tree paths and match A with B (thread 0)
    auto rematch = [&]() {
        flip_to_root(S, A);
        if (bout) flip_to_root(S, B);
        if (B >= 0) {
            S.mate[A] = B; S.ms[A] = a; S.mo[A] = b;
            S.mate[B] = A; S.ms[B] = b; S.mo[B] = a;
        } else {
            S.mate[A] = MATE_BOUNDARY; S.ms[A] = a; S.mo[A] = -1;
        }
    };
    if (T.tid() == 0) {
        rA = S.nroot[A];
        bout = B >= 0 && S.nd[B].label == 1;
        rB = bout ? S.nroot[B] : -3;
        if constexpr (NW == 1) rematch();
    }
    {
        // both roots in one broadcast (a block's broadcast is also its barrier)
        const unsigned long long pr = T.bcast64(((unsigned long long)(unsigned)rA << 32) | (unsigned)rB);
        rA = (int)(unsigned)(pr >> 32);
        rB = (int)(unsigned)(pr & 0xffffffffu);
    }
    if constexpr (NW == 1) {
        T.sync();
        for (int v = T.tid(); v < nhi; v += T.NT) {
            const int4 q = ld_nd(&S.nd[v]);
            if (q.w && q.y < 0 && q.z != 0 && (S.nroot[v] == rA || S.nroot[v] == rB)) {
                S.nd[v].label = 0; S.tpar[v] = -1; S.nroot[v] = -1;
            }
        }
    } else {
        // The two trees' nodes leave them (label and root cleared; a node's
        // tree parent is only read while it is in a tree, and is set again when
        // it joins one), while thread 0 rewrites the matches along the tree
        // paths, which reads tree parents and writes only mates: the two
        // overlap.  Independent loads first (one round trip per node).
        for (int v = T.tid(); v < nhi; v += T.NT) {
            const int4 q = ld_nd(&S.nd[v]);
            const int nr = S.nroot[v];
            if (q.w && q.y < 0 && q.z != 0 && (nr == rA || nr == rB)) { S.nd[v].label = 0; S.nroot[v] = -1; }
        }
        if (T.tid() == 0) rematch();
    }
    T.sync();
}

// Event (a): outer A touches frozen B (matched to C).  Thread 0 only.
__device__ void ev_grow(const Slab &S, int A, int a, int B, int b) {
    const int Cn = S.mate[B];
    S.nd[B].label = -1; S.tpar[B] = A; S.tps[B] = b; S.tpo[B] = a; S.nroot[B] = S.nroot[A];
    S.nd[Cn].label = 1; S.tpar[Cn] = B; S.tps[Cn] = S.ms[Cn]; S.tpo[Cn] = S.mo[Cn]; S.nroot[Cn] = S.nroot[A];
}

// Event (c): outer A, B in one tree form a blossom.  Every thread of the team calls.
template <int NW>
__device__ __noinline__ void ev_blossom(const Slab &S, Shot &C, int A, int a, int B, int b, Team<NW> T, int &nhi) {
    int N = -1, L = -1, Lroot = 0;
    if (T.tid() == 0) {
        int na = 0, nb = 0;
        for (int v = A; v >= 0 && na < 2 * C.nc; v = S.tpar[v]) S.tmpa[na++] = v;
        for (int v = B; v >= 0 && nb < 2 * C.nc; v = S.tpar[v]) S.tmpb[nb++] = v;
        while (na > 1 && nb > 1 && S.tmpa[na - 2] == S.tmpb[nb - 2]) { na--; nb--; }
        L = S.tmpa[na - 1];
        const int m = na + nb - 1;
        const int nf = S.ctr[C_NFREE];
        const int cb = S.ctr[C_CCOUNT];
        if (L != S.tmpb[nb - 1] || nf <= 0 || cb + m > C.cc) {
            S.ctr[C_ERR] |= (L != S.tmpb[nb - 1]) ? ERR_INTERNAL : ERR_CAP;
        } else {
            N = S.freel[nf - 1];
            S.ctr[C_NFREE] = nf - 1;
            S.ctr[C_CCOUNT] = cb + m;
            int i = 0;
            S.cnode[cb + i++] = L;
            for (int j = na - 2; j >= 0; j--) S.cnode[cb + i++] = S.tmpa[j];
            for (int j = 0; j <= nb - 2; j++) S.cnode[cb + i++] = S.tmpb[j];
            const int ia = na - 1;
            int ml = INT_MAX;
            for (int j = 0; j < m; j++) {
                const int x = S.cnode[cb + j], z = S.cnode[cb + (j + 1) % m];
                if (j < ia) { S.cs[cb + j] = S.tpo[z]; S.co[cb + j] = S.tps[z]; }
                else if (j == ia) { S.cs[cb + j] = a; S.co[cb + j] = b; }
                else { S.cs[cb + j] = S.tps[x]; S.co[cb + j] = S.tpo[x]; }
                ml = min(ml, S.minleaf[x]);
            }
            S.nd[N] = NRec{0, -1, 1, 1};
            S.tpar[N] = S.tpar[L]; S.tps[N] = S.tps[L]; S.tpo[N] = S.tpo[L];
            S.mate[N] = S.mate[L]; S.ms[N] = S.ms[L]; S.mo[N] = S.mo[L];
            Lroot = (S.nroot[L] == L);
            S.nroot[N] = Lroot ? N : S.nroot[L];
            S.minleaf[N] = ml; S.cbeg[N] = cb; S.clen[N] = m;
            for (int j = 0; j < m; j++) S.nd[S.cnode[cb + j]].bpar = N;
        }
    }
    {
        // N, L and whether L was its tree's root in one broadcast (ids < 2^18)
        const unsigned hi = L >= 0 ? ((unsigned)L | ((unsigned)Lroot << 30)) : 0xffffffffu;
        const unsigned long long pk = T.bcast64(((unsigned long long)hi << 32) | (unsigned)N);
        N = (int)(unsigned)(pk & 0xffffffffu);
        const unsigned h = (unsigned)(pk >> 32);
        L = h == 0xffffffffu ? -1 : (int)(h & 0x3fffffffu);
        Lroot = h == 0xffffffffu ? 0 : (int)((h >> 30) & 1u);
    }
    if constexpr (NW == 1) T.sync();
    if (N < 0) return;
    nhi = max(nhi, N + 1);
    for (int v = T.tid(); v < nhi; v += T.NT) {
        if constexpr (NW == 1) {
            const int4 q = ld_nd(&S.nd[v]);
            if (!q.w || q.y >= 0 || v == N) continue;
            const int tp = S.tpar[v];
            if (tp >= 0 && S.nd[tp].bpar == N) S.tpar[v] = N;
            const int mt = S.mate[v];
            if (mt >= 0 && S.nd[mt].bpar == N) S.mate[v] = N;
            if (Lroot && S.nroot[v] == L) S.nroot[v] = N;
        } else {
            // independent loads first, the parents' blossom pointers after
            const int4 q = ld_nd(&S.nd[v]);
            const int al = q.w, bp = q.y, tp = S.tpar[v], mt = S.mate[v], nr = S.nroot[v];
            if (!al || bp >= 0 || v == N) continue;
            const int btp = tp >= 0 ? S.nd[tp].bpar : -1, bmt = mt >= 0 ? S.nd[mt].bpar : -1;
            if (btp == N) S.tpar[v] = N;
            if (bmt == N) S.mate[v] = N;
            if (Lroot && nr == L) S.nroot[v] = N;
        }
    }
    for (int s = T.tid(); s < C.K; s += T.NT) {
        const int tp = S.src[s].stop;
        if (tp != N && S.nd[tp].bpar == N) S.src[s].stop = N;
    }
    T.sync();
}

// Event (d): inner blossom B with zero dual shatters.  Every thread of the team calls.
template <int NW>
__device__ __noinline__ void ev_shatter(const Slab &S, Shot &C, int B, Team<NW> T) {
    for (int s = T.tid(); s < C.K; s += T.NT)
        if (S.src[s].stop == B) {
            const int c = child_of(S, B, s);
            if (c >= 0) S.src[s].stop = c; else atomicOr(&S.ctr[C_ERR], ERR_INTERNAL);
        }
    T.sync();
    if (T.tid() == 0) {
        const int m = S.clen[B], cb = S.cbeg[B];
        const int P = S.tpar[B], Cn = S.mate[B];
        const int xp = S.tps[B] >= 0 ? child_of(S, B, S.tps[B]) : -1;
        const int xc = S.ms[B] >= 0 ? child_of(S, B, S.ms[B]) : -1;
        int ip = -1, ic = -1;
        for (int j = 0; j < m; j++) {
            if (S.cnode[cb + j] == xp) ip = j;
            if (S.cnode[cb + j] == xc) ic = j;
        }
        if (ip < 0 || ic < 0 || Cn < 0) {
            S.ctr[C_ERR] |= ERR_INTERNAL;
        } else {
            const int rootB = S.nroot[B];
            for (int j = 0; j < m; j++) S.nd[S.cnode[cb + j]].bpar = -1;
            const int fwd = ((ic - ip) % m + m) % m;
            const int dir = (fwd % 2 == 0) ? 1 : -1;
            const int L = dir > 0 ? fwd : m - fwd;
            int prev = -1;
            for (int j = 0; j <= L; j++) {
                const int idx = ((ip + dir * j) % m + m) % m;
                const int q = S.cnode[cb + idx];
                S.nd[q].label = (j % 2 == 0) ? -1 : 1;
                S.nroot[q] = rootB;
                if (j == 0) {
                    S.tpar[q] = P; S.tps[q] = S.tps[B]; S.tpo[q] = S.tpo[B];
                } else {
                    const int pidx = ((ip + dir * (j - 1)) % m + m) % m;
                    int self, other;
                    if (dir > 0) { self = S.co[cb + pidx]; other = S.cs[cb + pidx]; }
                    else { self = S.cs[cb + idx]; other = S.co[cb + idx]; }
                    S.tpar[q] = prev; S.tps[q] = self; S.tpo[q] = other;
                    if (j % 2 == 1) {
                        S.mate[q] = prev; S.ms[q] = self; S.mo[q] = other;
                        S.mate[prev] = q; S.ms[prev] = other; S.mo[prev] = self;
                    }
                }
                prev = q;
            }
            const int qL = prev;
            S.mate[qL] = Cn; S.ms[qL] = S.ms[B]; S.mo[qL] = S.mo[B];
            S.mate[Cn] = qL; S.tpar[Cn] = qL;
            const int rem = m - 1 - L;
            for (int j = 1; j <= rem; j += 2) {
                const int i1 = ((ic + dir * j) % m + m) % m;
                const int i2 = ((ic + dir * (j + 1)) % m + m) % m;
                const int x = S.cnode[cb + i1], z = S.cnode[cb + i2];
                int lx, lz;
                if (dir > 0) { lx = S.cs[cb + i1]; lz = S.co[cb + i1]; }
                else { lx = S.co[cb + i2]; lz = S.cs[cb + i2]; }
                S.nd[x].label = 0; S.nd[z].label = 0;
                S.tpar[x] = -1; S.tpar[z] = -1;
                S.nroot[x] = -1; S.nroot[z] = -1;
                S.mate[x] = z; S.ms[x] = lx; S.mo[x] = lz;
                S.mate[z] = x; S.ms[z] = lz; S.mo[z] = lx;
            }
            S.nd[B].alive = 0; S.tpar[B] = -1; S.mate[B] = MATE_NONE; S.nd[B].y = 0; S.clen[B] = 0;
            const int nf = S.ctr[C_NFREE];
            S.freel[nf] = B;
            S.ctr[C_NFREE] = nf + 1;
        }
    }
    T.sync();
}

// Fresh growing root for source s.
__device__ __forceinline__ void make_root(const Slab &S, int s) {
    S.nd[s] = NRec{0, -1, 1, 1}; S.src[s].srad = 0;
    S.tpar[s] = -1; S.mate[s] = MATE_NONE; S.nroot[s] = s; S.src[s].stop = s; S.src[s].inplay = 1;
}

enum { RUN_OK = 0, RUN_NOSOL = 1, RUN_BUDGET = 2, RUN_CAP = 3, RUN_INTERNAL = 4 };

// Event loop over the sources with inplay[s] = 1, from t = 0 (SI S1).
template <int NW>
__device__ int run_matcher(const Slab &S, Shot &C, Team<NW> &T, int &nhi) {
    C.t = 0;
    for (;;) {
        if (++C.events > C.max_events) return RUN_BUDGET;
        if (C.deadline && (C.events & 63) == 0) {
            int late = 0;
            if (T.tid() == 0) late = now_ns() > C.deadline;
            if (T.bcast(late)) return RUN_BUDGET;
        }
        unsigned long long best = EMPTY64;
        int flags = 0;   // bit 0: a growing region exists, bit 1: inconsistent state
        unsigned inner_leaf_min = INT_MAX;
        auto src_item = [&](int s) {
            // independent loads first, one dependent load (the label) after
            const int4 r = ld_src(&S.src[s]);
            const int ip = rec_inplay(r), A = r.x, rad = r.y, exh = rec_sexh(r), sR = r.z;
            const unsigned long long bb = ldr(&S.sbnd[s]);
            if (!ip) return;
            const int lab = S.nd[A].label;
            if (lab == 1) {
                flags |= 1;
                if (!exh) {
                    // due when Rad(s) + L would pass the explored radius; a region that
                    // just started growing (or was never explored) is due at once
                    const int ahead = sR - C.L + 1 - rad;
                    best = min(best, ev_key(C.t + (ahead > 0 ? ahead : 0), EV_EXTEND, s, 0));
                }
                if (bb != EMPTY64) {
                    const int bd = (int)(bb >> 32);
                    if (bd < rad) flags |= 2;
                    else best = min(best, ev_key(C.t + (bd - rad), EV_BOUNDARY, s, ID_MAX));
                }
            } else if (lab == -1 && A == s) {
                inner_leaf_min = min(inner_leaf_min, (unsigned)S.nd[s].y);
            }
        };
        auto pair_item = [&](int i) {
            int a, b, pv;
            if constexpr (NW == 1) {
                unsigned long long k;
                ld_ent(&S.pt[S.plist[i]], k, pv);
                a = (int)(k >> 32); b = (int)(unsigned)(k & 0xffffffffu);
            } else {   // the pair's record: one round trip less
                const int4 pq = ld_pr(&S.pr[i]);
                a = pq.x; b = pq.y; pv = pq.z;
                if (a < 0) return;
            }
            const int4 qa = ld_src(&S.src[a]), qb = ld_src(&S.src[b]);
            const int ia = rec_inplay(qa), ib = rec_inplay(qb), A = qa.x, B = qb.x;
            const int ra = qa.y, rb = qb.y;
            if (!ia || !ib || A == B) return;
            const int r = S.nd[A].label + S.nd[B].label;
            if (r <= 0) return;
            const int gap = pv - ra - rb;
            if (gap < 0 || gap % r) { flags |= 2; return; }
            best = min(best, ev_key(C.t + gap / r, EV_COLLIDE, a, b));
        };
        auto node_item = [&](int v) {
            const int4 q = ld_nd(&S.nd[v]);
            if constexpr (NW == 1) {
                if (q.w && q.y < 0 && q.z == -1) best = min(best, ev_key(C.t + q.x, EV_IMPLODE, S.minleaf[v], 0));
            } else {
                const int ml = S.minleaf[v];
                if (q.w && q.y < 0 && q.z == -1) best = min(best, ev_key(C.t + q.x, EV_IMPLODE, ml, 0));
            }
        };
        const int np = ldr(&S.ctr[C_NPAIRS]);
        if constexpr (NW == 1) {
            for (int s = T.tid(); s < C.K; s += T.NT) src_item(s);
            for (int i = T.tid(); i < np; i += T.NT) pair_item(i);
            for (int v = C.K + T.tid(); v < nhi; v += T.NT) node_item(v);
        } else {
            // one strided pass over sources, pairs and blossoms together, so
            // every thread of the block gets the same number of items
            const int n1 = C.K, n2 = C.K + np, n3 = np + nhi;
            for (int j = T.tid(); j < n3; j += T.NT) {
                if (j < n1) src_item(j);
                else if (j < n2) pair_item(j - n1);
                else node_item(j - np);
            }
        }
        // a block resets the EXTEND list counter ahead of the reduction's
        // barrier (nothing uses it between ball extensions)
        if constexpr (NW > 1) {
            if (T.tid() == 0) S.ctr[C_WL] = 0;
        }
        T.reduce_ev(best, flags, inner_leaf_min);
        if (flags & 2) return RUN_INTERNAL;
        if (!(flags & 1)) return RUN_OK;
        if (best == EMPTY64) return RUN_NOSOL;
        const long long tn = (long long)(best >> 38);
        const int kind = (int)((best >> 36) & 3);
        const int lo = (int)((best >> 18) & ID_MAX);
        const int hi = (int)(best & ID_MAX);
        if (tn >= T_MAX) return RUN_CAP;
        const int dt = (int)(tn - C.t);
        if ((unsigned)dt > inner_leaf_min) return RUN_INTERNAL;
        if (dt > 0) {
            for (int v = T.tid(); v < nhi; v += T.NT) {
                if constexpr (NW == 1) {
                    const int4 q = ld_nd(&S.nd[v]);
                    if (q.w && q.y < 0 && q.z != 0) S.nd[v].y = q.x + q.z * dt;
                } else {
                    const int4 q = ld_nd(&S.nd[v]);
                    if (q.w && q.y < 0 && q.z != 0) S.nd[v].y = q.x + q.z * dt;
                }
            }
            for (int s = T.tid(); s < C.K; s += T.NT) {
                const int4 r = ld_src(&S.src[s]);
                if (rec_inplay(r)) S.src[s].srad = r.y + S.nd[r.x].label * dt;
            }
        }
        C.t = tn;
        if (kind == EV_EXTEND) {
            C.nx++;
        } else {
            C.nm++;
            if (tn <= C.tcut) C.ncut++;
            C.tlast = (int)tn;
        }
        // The dual update above writes y and srad only.  In a block, the next
        // barrier is the one each step below starts with (EXTEND reads the radii
        // after it; the matcher steps read or write no radius before theirs);
        // one warp keeps its barrier here.
        if constexpr (NW == 1) T.sync();
        if (kind == EV_EXTEND) {
            // every growing region that reached its explored radius now.  In a
            // block the counter is already zero, and each thread reads only the
            // radii it updated itself (same striding as the dual update)
            if constexpr (NW == 1) {
                if (T.tid() == 0) S.ctr[C_WL] = 0;
                T.sync();
            }
            for (int s = T.tid(); s < C.K; s += T.NT) {
                const int4 r = ld_src(&S.src[s]);
                const int rad = r.y;
                if (rec_inplay(r) && !rec_sexh(r) && S.nd[r.x].label == 1 && r.z - C.L + 1 - rad <= 0) {
                    const int k = atomicAdd(&S.ctr[C_WL], 1);
                    S.xsrc[k] = s;
                    S.xR[k] = max(r.z + C.band, rad + C.L + C.band);
                }
            }
            T.sync();
            // after the barrier the counter stays unchanged until extend_many's
            // own first barrier: every thread reads the same count
            if constexpr (NW == 1) extend_many(S, C, T.bcast(ldr(&S.ctr[C_WL])), T);
            else extend_many(S, C, ldr(&S.ctr[C_WL]), T);
        } else if (kind == EV_IMPLODE) {
            // the blossom is read by every thread before any thread's shatter
            // loop rewrites the stop pointers
            const int B = S.src[lo].stop;
            if constexpr (NW > 1) T.sync();
            ev_shatter(S, C, B, T);
        } else if (kind == EV_BOUNDARY) {
            ev_augment(S, C, S.src[lo].stop, lo, -1, -1, T, nhi);
        } else {
            int a = lo, b = hi;
            int A = S.src[a].stop, B = S.src[b].stop;
            if (S.nd[A].label != 1) { int t = A; A = B; B = t; t = a; a = b; b = t; }
            const int lb = S.nd[B].label;
            // 0 blossom, 1 augment, 2 grow, 3 inconsistent
            int act = 3;
            if (lb == 1) act = S.nroot[A] == S.nroot[B] ? 0 : 1;
            else if (lb == 0 && S.mate[B] == MATE_BOUNDARY) act = 1;
            else if (lb == 0 && S.mate[B] >= 0) act = 2;
            // every thread has read the state it dispatches on before any
            // thread changes it
            if constexpr (NW > 1) T.sync();
            if (act == 0) ev_blossom(S, C, A, a, B, b, T, nhi);
            else if (act == 1) ev_augment(S, C, A, a, B, b, T, nhi);
            else if (act == 2) {
                if (T.tid() == 0) ev_grow(S, A, a, B, b);
                T.sync();
            } else {
                return RUN_INTERNAL;
            }
        }
        // the error word is written only before the barrier that ends each
        // step above and after the next event search's barrier, so every
        // thread reads the same value here
        const int err = ldr(&S.ctr[C_ERR]);
        if (err) return (err & ERR_INTERNAL) ? RUN_INTERNAL : RUN_CAP;
    }
}

// Canonical path observable from source s (its Dijkstra tree) to vertex x at
// distance dx: predecessor = lowest edge id among tight edges.  Every thread
// of the team calls.
template <int NW>
__device__ unsigned long long path_obs(const Slab &S, Shot &C, int s, int x, int dx, Team<NW> &T) {
    const DGraph &g = C.g;
    for (int n = 0; n < 1 << 16; n++) {
        const int more = S.src[s].sR < dx && !S.src[s].sexh && !ldr(&S.ctr[C_ERR]);
        if (!T.bcast(more)) break;
        extend_one(S, C, s, T);
    }
    // a ball that outgrew the tables: the attempt is retried with larger ones
    if (T.bcast(ldr(&S.ctr[C_ERR]))) return 0;
    unsigned long long o = 0;
    const int src = S.svtx[s];
    int cur = x, dcur = dx;
    for (int n = 0; n < 1 << 22 && cur != src; n++) {
        const int r0 = __ldg(g.row + cur), r1 = __ldg(g.row + cur + 1);
        unsigned long long best = EMPTY64;
        for (int j = r0 + T.tid(); j < r1; j += T.NT) {
            SlotV sl = load_slot(g, j);
            if (sl.nbr < 0) continue;
            const int dy = ht_get(S, C, sl.nbr, s);
            if (dy != INF32 && dy + sl.w == dcur)
                best = min(best, ((unsigned long long)(unsigned)__ldg(g.seid + j) << 32) | (unsigned)sl.nbr);
        }
        best = T.min64(best);
        if (best == EMPTY64) { if (T.tid() == 0) S.ctr[C_ERR] |= ERR_INTERNAL; break; }
        const int e = (int)(best >> 32);
        o ^= __ldg(g.eobs + e);
        cur = (int)(unsigned)(best & 0xffffffffu);
        dcur = ht_get(S, C, cur, s);
    }
    T.sync();
    return o;
}

// Expand the final matching into leaf-level pairs (tmpa[i], tmpb[i]; tmpb = -1
// for a boundary match) and accumulate weight (internal units) and obs.
template <int NW>
__device__ __noinline__ void trace(const Slab &S, Shot &C, Team<NW> T, int nhi, long long &wint,
                                   unsigned long long &obs) {
    // matched top-level nodes, team-parallel: each match appends its leaf pair
    // and queues the blossoms on either side for expansion (stack seeds)
    if (T.tid() == 0) { S.ctr[C_TNP] = 0; S.ctr[C_TNX] = 0; }
    T.sync();
    int *stk = S.stk;
    for (int v = T.tid(); v < nhi; v += T.NT) {
        if (!S.nd[v].alive || S.nd[v].bpar >= 0) continue;
        const int mt = S.mate[v];
        if (mt == MATE_BOUNDARY) {
            const int k = agg_inc(&S.ctr[C_TNP], T.lane);
            S.tmpa[k] = S.ms[v]; S.tmpb[k] = -1;
            if (v >= C.K) { const int x = atomicAdd(&S.ctr[C_TNX], 1); stk[2 * x] = v; stk[2 * x + 1] = S.ms[v]; }
        } else if (mt >= 0 && v < mt) {
            const int k = agg_inc(&S.ctr[C_TNP], T.lane);
            S.tmpa[k] = S.ms[v]; S.tmpb[k] = S.mo[v];
            if (v >= C.K) { const int x = atomicAdd(&S.ctr[C_TNX], 1); stk[2 * x] = v; stk[2 * x + 1] = S.ms[v]; }
            if (mt >= C.K) { const int x = atomicAdd(&S.ctr[C_TNX], 1); stk[2 * x] = mt; stk[2 * x + 1] = S.mo[v]; }
        }
    }
    T.sync();
    int np = ldr(&S.ctr[C_TNP]);
    if (T.tid() == 0) {
        // blossoms: the child holding the externally matched leaf keeps that
        // match, the other children pair up along the cycle
        const int stk_cap = 4 * C.nc + 60;
        int sp = 2 * ldr(&S.ctr[C_TNX]);
        while (sp > 0) {
            const int ext = stk[--sp];
            const int node = stk[--sp];
            if (node < C.K) continue;
            const int m = S.clen[node], cb = S.cbeg[node];
            const int c0 = ext >= 0 ? child_of(S, node, ext) : -1;
            if (c0 < 0 || m <= 0) { S.ctr[C_ERR] |= ERR_INTERNAL; break; }
            int i0 = 0;
            for (int j = 0; j < m; j++) if (S.cnode[cb + j] == c0) i0 = j;
            if (sp + 2 * m + 2 > stk_cap || np + m > 2 * C.nc) { S.ctr[C_ERR] |= ERR_CAP; break; }
            stk[sp++] = c0; stk[sp++] = ext;
            for (int j = 1; j < m; j += 2) {
                const int i1 = (i0 + j) % m, i2 = (i0 + j + 1) % m;
                const int lx = S.cs[cb + i1], lz = S.co[cb + i1];
                S.tmpa[np] = lx; S.tmpb[np] = lz; np++;
                stk[sp++] = S.cnode[cb + i1]; stk[sp++] = lx;
                stk[sp++] = S.cnode[cb + i2]; stk[sp++] = lz;
            }
        }
    }
    np = T.bcast(np);
    T.sync();
    if (T.tid() == 0) S.ctr[C_TNP] = np;   // leaf pairs in tmpa / tmpb, read by commit_trace
    long long w = 0;
    unsigned long long o = 0;
    for (int i = T.tid(); i < np; i += T.NT) {
        const int a = S.tmpa[i], b = S.tmpb[i];
        if (a < 0 || a >= C.K || b >= C.K) { set_err(S, ERR_INTERNAL); continue; }
        if (b < 0) {
            const unsigned long long bb = ldr(&S.sbnd[a]);
            if (bb == EMPTY64) { set_err(S, ERR_INTERNAL); continue; }
            w += (long long)(bb >> 32);
            o ^= __ldg(C.g.eobs + (int)(unsigned)(bb & 0xffffffffu));
        } else {
            const int d = pair_get(S, C, a, b);
            if (d == INF32) { set_err(S, ERR_INTERNAL); continue; }
            w += d;
        }
    }
    w = T.sum64(w);
    o = T.xor64(o);
    if (C.g.internal_obs && !T.bcast(ldr(&S.ctr[C_ERR]))) {
        // detector-detector edges carry observables: walk the canonical paths
        for (int i = 0; i < np; i++) {
            const int a = S.tmpa[i], b = S.tmpb[i];
            if (b < 0) {
                const unsigned long long bb = ldr(&S.sbnd[a]);
                const int e = (int)(unsigned)(bb & 0xffffffffu);
                const int2 ue = __ldg(C.g.eend + e);
                o ^= path_obs(S, C, a, ue.x, (int)(bb >> 32) - ue.y, T);
            } else {
                const int lo = min(a, b), hi = max(a, b);
                o ^= path_obs(S, C, lo, S.svtx[hi], pair_get(S, C, lo, hi), T);
            }
        }
    }
    wint = w;
    obs = o;
    T.sync();
}

__device__ __forceinline__ bool in_commit(const DGraph &g, int v) {
    return (__ldg(g.commit + (v >> 5)) >> (v & 31)) & 1u;
}

// Canonical path from source s's vertex to vertex x at distance dx (the path
// of path_obs): the XOR of the observables of its edges that touch the commit
// region; each such edge with its other endpoint outside the region flips that
// endpoint in `carry` (thread 0 writes).  Every thread of the team calls.
template <int NW>
__device__ unsigned long long path_commit(const Slab &S, Shot &C, int s, int x, int dx, Team<NW> &T,
                                          unsigned *carry) {
    const DGraph &g = C.g;
    for (int n = 0; n < 1 << 16; n++) {
        const int more = S.src[s].sR < dx && !S.src[s].sexh && !ldr(&S.ctr[C_ERR]);
        if (!T.bcast(more)) break;
        extend_one(S, C, s, T);
    }
    // a ball that outgrew the tables: the attempt is retried with larger ones
    if (T.bcast(ldr(&S.ctr[C_ERR]))) return 0;
    unsigned long long o = 0;
    const int src = S.svtx[s];
    int cur = x, dcur = dx;
    for (int n = 0; n < 1 << 22 && cur != src; n++) {
        const int r0 = __ldg(g.row + cur), r1 = __ldg(g.row + cur + 1);
        unsigned long long best = EMPTY64;
        for (int j = r0 + T.tid(); j < r1; j += T.NT) {
            SlotV sl = load_slot(g, j);
            if (sl.nbr < 0) continue;
            const int dy = ht_get(S, C, sl.nbr, s);
            if (dy != INF32 && dy + sl.w == dcur)
                best = min(best, ((unsigned long long)(unsigned)__ldg(g.seid + j) << 32) | (unsigned)sl.nbr);
        }
        best = T.min64(best);
        if (best == EMPTY64) { if (T.tid() == 0) S.ctr[C_ERR] |= ERR_INTERNAL; break; }
        const int e = (int)(best >> 32);
        const int nxt = (int)(unsigned)(best & 0xffffffffu);
        const bool ci = in_commit(g, cur), ni = in_commit(g, nxt);
        if (ci || ni) {
            o ^= __ldg(g.eobs + e);
            if (ci != ni && T.tid() == 0) {
                const int out = ci ? nxt : cur;
                carry[out >> 5] ^= 1u << (out & 31);
            }
        }
        cur = nxt;
        dcur = ht_get(S, C, cur, s);
    }
    T.sync();
    return o;
}

// Sliding-window commit of a decoded shot (the leaf pairs left by trace): the
// correction is the union of the canonical matching paths (and boundary
// edges); every edge that touches the graph's commit region is committed.
// Returns the committed observable; the shot's carry row receives the
// detectors outside the region flipped by committed edges.  Every thread of
// the team calls.
template <int NW>
__device__ __noinline__ unsigned long long commit_trace(const Slab &S, Shot &C, Team<NW> T, unsigned *carry) {
    const DGraph &g = C.g;
    for (int w = T.tid(); w < g.words; w += T.NT) carry[w] = 0u;
    T.sync();
    const int np = T.bcast(ldr(&S.ctr[C_TNP]));
    unsigned long long o = 0;
    for (int i = 0; i < np; i++) {
        if (T.bcast(ldr(&S.ctr[C_ERR]))) break;
        const int a = S.tmpa[i], b = S.tmpb[i];
        if (b < 0) {
            const unsigned long long bb = ldr(&S.sbnd[a]);
            const int e = (int)(unsigned)(bb & 0xffffffffu);
            const int2 ue = __ldg(g.eend + e);
            if (in_commit(g, ue.x)) o ^= __ldg(g.eobs + e);   // the boundary edge itself
            o ^= path_commit(S, C, a, ue.x, (int)(bb >> 32) - ue.y, T, carry);
        } else {
            const int lo = min(a, b), hi = max(a, b);
            o ^= path_commit(S, C, lo, S.svtx[hi], pair_get(S, C, lo, hi), T, carry);
        }
    }
    T.sync();
    return o;
}

// Per-shot counters; the tables themselves are already empty (release_tables).
template <int NW>
__device__ void clear_tables(const Slab &S, const Shot &C, Team<NW> &T) {
    for (int i = T.tid(); i < C_TOTAL; i += T.NT) S.ctr[i] = 0;
    T.sync();
}

// Return the explored and pair tables to empty: the slots recorded in the band
// lists (every explored entry) and the pair list (every pair), or with `all`
// the whole region of this attempt's table sizes.
template <int NW>
__device__ __noinline__ void release_tables(const Slab &S, const Shot &C, Team<NW> T, bool all) {
    T.sync();
    const HEnt e = HEnt{EMPTY64, -1, -1};
    const PRec pe = PRec{-1, -1, ~0u, -1};
    if (all) {
        for (unsigned i = T.tid(); i <= C.hmask; i += T.NT) S.ht[i] = e;
        for (unsigned i = T.tid(); i <= C.pmask; i += T.NT) S.pt[i] = e;
        if constexpr (NW > 1)
            for (unsigned i = T.tid(); i <= (C.pmask >> 1); i += T.NT) S.pr[i] = pe;
    } else {
        const int ne = ldr(&S.ctr[C_ECOUNT]), np = ldr(&S.ctr[C_NPAIRS]);
        for (int i = T.tid(); i < ne; i += T.NT) S.ht[S.ent[i] & C.hmask] = e;
        if constexpr (NW == 1) {
            for (int i = T.tid(); i < np; i += T.NT) S.pt[S.plist[i] & C.pmask] = e;
        } else {
            for (int i = T.tid(); i < np; i += T.NT) {
                const int sl = S.pr[i].slot;
                if (sl >= 0) S.pt[sl & C.pmask] = e;
                S.pr[i] = pe;
            }
        }
    }
    T.sync();
}

__device__ __forceinline__ unsigned next_pow2(unsigned x) {
    x--; x |= x >> 1; x |= x >> 2; x |= x >> 4; x |= x >> 8; x |= x >> 16;
    return x + 1;
}

// Compact the set bits of the shot's syndrome row into S.svtx; returns K
// (or -1 when K exceeds kcap).  One warp.
__device__ int load_defects(const Slab &S, const DGraph &g, const unsigned *row, int kcap, int wcap, int lane) {
    int K = 0;
    const int nvec = g.words >> 2;
    const uint4 *rv = reinterpret_cast<const uint4 *>(row);
    for (int base = 0; base < nvec; base += WS) {
        const int i = base + lane;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (i < nvec) v = __ldg(rv + i);
        unsigned wv[4] = {v.x, v.y, v.z, v.w};
        // drop padding bits beyond n
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int bit0 = (i * 4 + q) * 32;
            if (bit0 >= g.n) wv[q] = 0;
            else if (bit0 + 32 > g.n) wv[q] &= (1u << (g.n - bit0)) - 1u;
        }
        int c = __popc(wv[0]) + __popc(wv[1]) + __popc(wv[2]) + __popc(wv[3]);
        int incl = c;
#pragma unroll
        for (int o = 1; o < WS; o <<= 1) {
            int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(FULL, incl, WS - 1);
        int pos = K + incl - c;
        if (i < nvec && i * 4 + 3 < wcap) {
            S.wcum[i * 4 + 0] = pos;
            S.wcum[i * 4 + 1] = pos + __popc(wv[0]);
            S.wcum[i * 4 + 2] = pos + __popc(wv[0]) + __popc(wv[1]);
            S.wcum[i * 4 + 3] = pos + __popc(wv[0]) + __popc(wv[1]) + __popc(wv[2]);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            unsigned bits = wv[q];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                if (pos < kcap) S.svtx[pos] = (i * 4 + q) * 32 + b;
                pos++;
            }
        }
        K += total;
    }
    __syncwarp();
    return K > kcap ? -1 : K;
}

constexpr int LB_CAP = 64;   // vertices one lane holds while exploring one event

// Lane-local bounded Dijkstra from event s to radius Rb (one lane, no shared
// tables): records every other event within Rb through pair_upsert (from the
// lower-ranked end only) and the canonical boundary candidate of s.  Returns
// the number of vertices settled, or -1 if more than LB_CAP lie within Rb.
template <bool REC>
__device__ __noinline__ int local_ball(const Slab &S, const Shot &C, int s, int Rb) {
    const DGraph &g = C.g;
    int vv[LB_CAP], dd[LB_CAP];
    unsigned long long fin = 0;   // settled flags
    const int src = S.svtx[s];
    int n = 1;
    vv[0] = src;
    dd[0] = 0;
    unsigned long long bbest = EMPTY64;
    int settled = 0;
    for (int it = 0; it < LB_CAP; it++) {
        int bi = -1, bd = INT_MAX;
        for (int i = 0; i < n; i++)
            if (!((fin >> i) & 1ull) && dd[i] < bd) { bd = dd[i]; bi = i; }
        if (bi < 0) break;
        fin |= 1ull << bi;
        settled++;
        const int x = vv[bi], dx = bd;
        if (x != src && is_defect(C, x)) {
            const int f = rank_of(S, C, x);
            if (f > s) pair_upsert<REC>(S, C, s, f, dx);
        }
        const int r0 = __ldg(g.row + x), r1 = __ldg(g.row + x + 1);
        for (int j = r0; j < r1; j++) {
            const SlotV sl = load_slot(g, j);
            const int nd = dx + sl.w;
            if (sl.nbr < 0) {
                const unsigned long long c = ((unsigned long long)(unsigned)nd << 32) | (unsigned)sl.eid;
                bbest = c < bbest ? c : bbest;
                continue;
            }
            if (nd > Rb) continue;
            int k = 0;
            while (k < n && vv[k] != sl.nbr) k++;
            if (k < n) {
                if (!((fin >> k) & 1ull) && nd < dd[k]) dd[k] = nd;
            } else {
                if (n == LB_CAP) return -1;
                vv[n] = sl.nbr;
                dd[n] = nd;
                n++;
            }
        }
    }
    atomicMin(&S.sbnd[s], bbest);
    return settled;
}

// Level-1 neighbourhoods by enumeration, for graphs in which a path of length
// <= Rb has at most two edges (DGraph::hop2): every event reached from event s
// by a path of one or two edges of length <= Rb is recorded through
// pair_upsert from the lower-ranked end (the minimum over those paths is the
// exact distance, since the shortest path has at most two edges), and the
// boundary candidates through s itself or a neighbour within Rb go to sbnd[s].
// Same records as local_ball's for every use: pairs within Rb exactly, and the
// canonical boundary contact whenever it lies within Rb / 2 (a longer contact
// is only an upper bound, refined by the flooder before a region can reach
// it).  One lane per (event, adjacency slot of the event), numbered by a warp
// prefix sum of the degrees; the warps of a team take 32 events each in turn.
// Every thread of the team calls (no team barrier inside).
template <int NW>
__device__ __noinline__ void level1_2hop(const Slab &S, const Shot &C, int Rb, const Team<NW> T) {
    const DGraph &g = C.g;
    const int lane = T.lane;
    for (int base = T.warp() * WS; base < C.K; base += T.NT) {
        const int s = base + lane;
        int src = -1, r0 = 0, deg = 0;
        if (s < C.K) {
            src = S.svtx[s];
            r0 = __ldg(g.row + src);
            deg = __ldg(g.row + src + 1) - r0;
        }
        int incl = deg;
        for (int o = 1; o < WS; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, WS - 1);
        const int excl = incl - deg;
        for (int t0 = 0; t0 < total; t0 += WS) {
            const int t = t0 + lane;
            int ow = 0;
            for (int step = WS / 2; step > 0; step >>= 1) {
                const int e = __shfl_sync(FULL, excl, ow + step);
                if (e <= t) ow += step;
            }
            const int osrc = __shfl_sync(FULL, src, ow);
            const int oj = __shfl_sync(FULL, r0 - excl, ow) + t;
            if (t >= total) continue;
            const int os = base + ow;
            const SlotV a = load_slot(g, oj);
            if (a.nbr < 0) {
                atomicMin(&S.sbnd[os], ((unsigned long long)(unsigned)a.w << 32) | (unsigned)a.eid);
                continue;
            }
            if (a.w > Rb) continue;
            if (is_defect(C, a.nbr)) {
                const int f = rank_of(S, C, a.nbr);
                if (f > os) pair_upsert<(NW > 1)>(S, C, os, f, a.w);
            }
            unsigned long long bbest = EMPTY64;
            const int q0 = __ldg(g.row + a.nbr), q1 = __ldg(g.row + a.nbr + 1);
            for (int k = q0; k < q1; k++) {
                const SlotV b = load_slot(g, k);
                const int nd = a.w + b.w;
                if (b.nbr < 0) {
                    const unsigned long long c = ((unsigned long long)(unsigned)nd << 32) | (unsigned)b.eid;
                    bbest = c < bbest ? c : bbest;
                    continue;
                }
                if (nd > Rb || b.nbr == osrc || !is_defect(C, b.nbr)) continue;
                const int f = rank_of(S, C, b.nbr);
                if (f > os) pair_upsert<(NW > 1)>(S, C, os, f, nd);
            }
            if (bbest != EMPTY64) atomicMin(&S.sbnd[os], bbest);
        }
    }
}

// Decode one shot with hash tables scaled by `scale`; returns QEC_SHOT_* or -1
// when the working set overflowed (retry with a larger scale).
// WIN: sliding-window mode (BatchArgs::carry set), compiled as its own kernel so
// that the ordinary kernel carries none of its code.
template <bool WIN, int NW>
__device__ int decode_attempt_body(const BatchArgs &A, const Slab &S, const DGraph &g, const unsigned *row,
                                   Team<NW> &T, unsigned scale, unsigned long long deadline, long long &w_out,
                                   unsigned long long &o_out, int *dg, Shot &C) {
    C.g = g;
    C.ec = A.caps.ec; C.wc = A.caps.wc; C.cc = A.caps.cc;
    C.band = max(g.wmax, 1) * max(A.band_factor, 1);
    C.events = 0;
    C.t = 0;
    C.deadline = deadline;
    C.row = row;
    C.L = max(g.wmax, (g.b1 + 1) / 2) + 1;
    C.nm = 0; C.ncut = 0; C.tcut = 0; C.tlast = 0; C.nx = 0;
    if (g.words > A.caps.wcap) return -2;
    int K = 0;
    if (T.warp() == 0) K = load_defects(S, g, row, A.caps.kc, A.caps.wcap, T.lane);
    K = T.bcast(K);
    T.sync();
    if (K < 0) return -2;
    C.K = K;
    C.max_events = min(A.max_events, 256LL * K + 4096);
    if (K == 0) {
        w_out = 0; o_out = 0;
        if (dg && T.tid() < QEC_DIAG_FIELDS) dg[T.tid()] = 0;   // no detection event: E_ideal = 0
        if constexpr (WIN)
            for (int w = T.tid(); w < g.words; w += T.NT) A.carry[(row - A.syn) + w] = 0u;
        return QEC_SHOT_OK;
    }
    if (K > ID_MAX - 1 || 2 * K + 8 > A.caps.nc) return -2;
    C.nc = min(A.caps.nc, 2 * K + 16);   // leaves + at most K blossoms alive at once
    // about 8 (rarely ~15) explored entries and 1 (at most ~2) pair per
    // detection event at the design point; the tables stay at most half full or
    // the shot is retried with larger ones
    const unsigned hs = min(next_pow2(max(128u, (unsigned)QEC_HT_FACTOR * (unsigned)K * scale)), (unsigned)A.caps.hc);
    const unsigned ps = min(next_pow2(max(64u, 4u * (unsigned)K * scale)), (unsigned)A.caps.phc);
    C.hmask = hs - 1;
    C.pmask = ps - 1;
    clear_tables(S, C, T);
    // sources, leaf nodes, free list
    int nhi = K;
    for (int s = T.tid(); s < K; s += T.NT) {
        S.src[s] = SRec{s, 0, -1, 0, 0, 0, 0}; S.scnt[s] = 0; S.sbeg[s] = 0;
        S.sbnd[s] = EMPTY64;
        S.nd[s] = NRec{0, -1, 0, 0}; S.tpar[s] = -1;
        S.mate[s] = MATE_NONE; S.nroot[s] = -1; S.minleaf[s] = s; S.clen[s] = 0;
    }
    const int nfree = C.nc - K;
    for (int i = T.tid(); i < nfree; i += T.NT) {
        const int v = C.nc - 1 - i;   // pop order: K, K+1, ...
        S.freel[i] = v;
        S.nd[v] = NRec{0, -1, 0, 0}; S.clen[v] = 0;
    }
    if (T.tid() == 0) { S.ctr[C_ECOUNT] = 0; S.ctr[C_NFREE] = nfree; }
    T.sync();
    // level-1 critical path (stopping time, event count), clusters, events
    // resolved at level 1, events of all level-1 runs
    int t1 = 0, e1 = 0, ncl1 = 0, nres1 = 0, ntot = 0;
    int gr = K;   // next level-1 cluster (its lowest event) that needs the event loop
    if (A.mode == QEC_MODE_HIERARCHICAL) {
        // ---- Algorithm 1, level 1: every event's neighbourhood within b_1 by a
        // lane-local Dijkstra (each lane its own events): pairs within b_1 with their
        // exact distance (found by reaching the other event's vertex) and the
        // canonical boundary candidate.  Events whose neighbourhood is too large for
        // the lane go through the team-wide flooder instead.
        bool any_big = false;
        if (g.hop2) {
            level1_2hop(S, C, g.b1, T);
        } else {
            for (int s = T.tid(); s < K; s += T.NT) {
                const int r = local_ball<(NW > 1)>(S, C, s, g.b1);
                if (r < 0) { S.cst0[s] = 1; any_big = true; } else S.cst0[s] = 0;
            }
        }
        T.sync();
        if (T.any(any_big)) {
            if (T.tid() == 0) {
                int k = 0;
                for (int s = 0; s < K; s++)
                    if (S.cst0[s]) { S.xsrc[k] = s; S.xR[k] = max(g.b1, C.band); k++; }
                S.ctr[C_WL] = k;
            }
            T.sync();
            extend_many(S, C, T.bcast(ldr(&S.ctr[C_WL])), T);
        }
        {
            const int err = T.bcast(ldr(&S.ctr[C_ERR]));
            if (err) return (err & ERR_INTERNAL) ? QEC_SHOT_INTERNAL : -1;
        }
        const int npairs = T.bcast(ldr(&S.ctr[C_NPAIRS]));
        // connected components of pairs within b_1: min-label propagation
        for (int s = T.tid(); s < K; s += T.NT) { S.comp[s] = s; S.cst0[s] = 0; S.cst1[s] = 0; S.cst2[s] = 0; }
        T.sync();
        for (int round = 0; round <= K; round++) {
            bool changed = false;
            for (int i = T.tid(); i < npairs; i += T.NT) {
                int a, b, pv;
                if (!pair_at<NW>(S, i, a, b, pv) || pv > g.b1) continue;
                const int la = ldr(&S.comp[a]), lb = ldr(&S.comp[b]);
                if (la != lb) {
                    const int m = min(la, lb);
                    atomicMin(&S.comp[a], m);
                    atomicMin(&S.comp[b], m);
                    changed = true;
                }
            }
            T.sync();
            if (!T.any(changed)) break;
        }
        for (int s = T.tid(); s < K; s += T.NT) {
            const int r = S.comp[s];
            atomicAdd(&S.cst0[r], 1);
            const unsigned long long bb = S.sbnd[s];
            if (bb != EMPTY64 && 2LL * (long long)(bb >> 32) <= (long long)g.b1) atomicOr(&S.cst1[r], 1);
        }
        T.sync();
        // pairs within d_1 inside a component; each such pair also names its
        // two events as each other's partner (xcur is free until the flooder
        // runs), which is the partner of an accepted two-event cluster
        for (int i = T.tid(); i < npairs; i += T.NT) {
            int a, b, pv;
            if (!pair_at<NW>(S, i, a, b, pv) || pv > g.d1) continue;
            if (S.comp[a] == S.comp[b]) {
                atomicAdd(&S.cst2[S.comp[a]], 1);
                S.xcur[a] = b;
                S.xcur[b] = a;
            }
        }
        T.sync();
        // ---- level-1 clusters: closed forms for isolated pairs / boundary singletons
        bool need_general = false;
        for (int s = T.tid(); s < K; s += T.NT) {
            const int r = S.comp[s];
            const int size = S.cst0[r];
            const bool ok = (long long)S.cst2[r] == (long long)size * (size - 1) / 2 &&
                            ((S.cst1[r] & 1) || size % 2 == 0);
            if (!ok) continue;
            if (size == 1) {
                const int bd = (int)(S.sbnd[s] >> 32);
                S.nd[s] = NRec{bd, -1, 0, 1}; S.src[s].srad = bd;
                S.mate[s] = MATE_BOUNDARY; S.ms[s] = s; S.mo[s] = -1; S.src[s].stop = s; S.nroot[s] = -1;
                t1 = max(t1, bd); ncl1++; nres1++;   // one boundary event at time bd
            } else if (size == 2) {
                // partner: the other member (its pair is the cluster's one pair
                // within d_1, recorded above)
                const int other = S.xcur[s];
                const int d = pair_get(S, C, s, other);
                const long long ba = (long long)(S.sbnd[s] >> 32), bo = (long long)(S.sbnd[other] >> 32);
                if (d / 2 <= ba && d / 2 <= bo) {
                    S.nd[s] = NRec{d / 2, -1, 0, 1}; S.src[s].srad = d / 2;
                    S.mate[s] = other; S.ms[s] = s; S.mo[s] = other; S.src[s].stop = s; S.nroot[s] = -1;
                    t1 = max(t1, d / 2); nres1++;   // one collision at time d/2
                    if (s < other) ncl1++;
                } else {
                    need_general = true;
                    atomicOr(&S.cst1[r], 2);   // solve with the event loop
                }
            } else {
                need_general = true;
                atomicOr(&S.cst1[r], 2);
            }
        }
        T.sync();
        t1 = T.maxi(t1);
        ncl1 = T.add(ncl1);
        nres1 = T.add(nres1);
        e1 = ncl1 > 0 ? 1 : 0;
        ntot = ncl1;
        need_general = T.any(need_general);
        gr = need_general ? 0 : K;
    }
    // ---- level-1 clusters without a closed form, one run each (from an empty
    // state apart from themselves), then the top level: every remaining event
    // from t = 0 with the stopped level-1 configurations present as frozen
    // regions (global mode: every event, from an empty state).  One call site
    // of the event loop serves both, which keeps the kernel's hot code small.
    for (int guard = 0; guard <= K + 1; guard++) {
        while (gr < K && (S.comp[gr] != gr || !(S.cst1[gr] & 2))) gr++;
        const bool top = gr >= K;
        if (top) {
            for (int s = T.tid(); s < K; s += T.NT) {
                if (S.nd[s].alive || S.src[s].stop != s) S.src[s].inplay = 1;   // stopped level-1 configuration
                else make_root(S, s);
            }
            C.ncut = 0;
            C.tcut = t1;
        } else {
            for (int s = T.tid(); s < K; s += T.NT)
                if (S.comp[s] == gr) make_root(S, s);
        }
        T.sync();
        C.nm = 0;
        C.tlast = 0;
        const int st = run_matcher(S, C, T, nhi);
        if (st != RUN_OK) {
            if (st == RUN_CAP) return -1;
            return st == RUN_NOSOL ? QEC_SHOT_NO_SOLUTION
                   : st == RUN_BUDGET ? QEC_SHOT_BUDGET_EXCEEDED : QEC_SHOT_INTERNAL;
        }
        if (top) break;
        for (int s = T.tid(); s < K; s += T.NT)
            if (S.comp[s] == gr) S.src[s].inplay = 0;
        T.sync();
        e1 = max(e1, C.nm); t1 = max(t1, C.tlast); ntot += C.nm; ncl1++; nres1 += S.cst0[gr];
        gr++;
    }
    long long wint = 0;
    unsigned long long ob = 0;
    trace(S, C, T, nhi, wint, ob);
    if constexpr (WIN) {   // sliding window: the committed part
        if (!T.bcast(ldr(&S.ctr[C_ERR]))) ob = commit_trace(S, C, T, A.carry + (row - A.syn));
    }
    const int err = T.bcast(ldr(&S.ctr[C_ERR]));
    if (err) return (err & ERR_INTERNAL) ? QEC_SHOT_INTERNAL : -1;
    w_out = wint / 2;
    o_out = ob;
    if (dg && T.tid() == 0) {
        // parallel event count over level 1 and the top level (Methods,
        // "Numerical evaluation"): the top run's events up to the level-1
        // critical-path time t1 overlap level 1, the rest extend it
        const int ntop = C.nm;
        dg[QEC_DIAG_E_IDEAL] = ntop > 0 ? max(e1, C.ncut) + ntop - C.ncut : e1;
        dg[QEC_DIAG_T_IDEAL] = ntop > 0 ? max(t1, C.tlast) : t1;
        dg[QEC_DIAG_EVENTS] = ntot + ntop;
        dg[QEC_DIAG_L1_CLUSTERS] = ncl1;
        dg[QEC_DIAG_L1_DEFECTS] = nres1;
        dg[QEC_DIAG_TOP_EVENTS] = ntop;
        dg[QEC_DIAG_BANDS] = C.nx;
        dg[QEC_DIAG_DEFECTS] = K;
    }
    return QEC_SHOT_OK;
}

// One decode attempt.  The explored and pair tables are empty (all-ones) on
// entry and are returned empty: after a successful shot only the slots listed
// in the band lists and the pair list are reset, after anything else the
// whole region the attempt could have used.
template <bool WIN, int NW>
__device__ int decode_attempt(const BatchArgs &A, const Slab &S, const DGraph &g, const unsigned *row, Team<NW> &T,
                              unsigned scale, unsigned long long deadline, long long &w_out,
                              unsigned long long &o_out, int *dg) {
    Shot C;
    C.hmask = 0;
    C.pmask = 0;
    const int st = decode_attempt_body<WIN, NW>(A, S, g, row, T, scale, deadline, w_out, o_out, dg, C);
    if (C.hmask) release_tables(S, C, T, st != QEC_SHOT_OK);
    return st;
}

// Detection events of a syndrome row (padding bits beyond n ignored).  One warp.
__device__ int count_defects(const DGraph &g, const unsigned *row, int lane) {
    int c = 0;
    for (int w = lane; w < g.words; w += WS) {
        unsigned v = __ldg(row + w);
        const int bit0 = w * 32;
        if (bit0 >= g.n) v = 0;
        else if (bit0 + 32 > g.n) v &= (1u << (g.n - bit0)) - 1u;
        c += __popc(v);
    }
    return (int)__reduce_add_sync(FULL, (unsigned)c);
}

template <bool WIN, int NW>
__device__ void decode_shot(const BatchArgs &A, const Slab &S, long long shot, Team<NW> &T,
                            unsigned long long deadline) {
    int gi = A.graph_of_shot ? A.graph_of_shot[shot] : 0;
    if (gi < 0 || gi >= A.num_graphs) gi = 0;
    const DGraph &g = A.g[gi];
    const long long off = A.syn_off ? A.syn_off[shot] : shot * (long long)g.words;
    const unsigned *row = A.syn + off;
    if constexpr (NW > 1) {
        // a shot below the split threshold goes to the team's first warp
        // alone (a team's barriers cost more than its lanes save there)
        if (A.team_split > 0) {
            int K = 0;
            if (T.warp() == 0) K = count_defects(g, row, T.lane);
            K = T.bcast(K);
            if (K < A.team_split) {
                if (T.warp() == 0) {
                    Team<1> T1;
                    T1.lane = T.lane;
                    decode_shot<WIN, 1>(A, S, shot, T1, deadline);
                }
                T.sync();
                return;
            }
        }
    }
    int status = -1;
    long long w = 0;
    unsigned long long o = 0;
    int *dg = A.diag_out ? A.diag_out + shot * QEC_DIAG_FIELDS : nullptr;
    for (unsigned scale = 1; scale <= 64 && status == -1; scale *= 4)
        status = decode_attempt<WIN, NW>(A, S, g, row, T, scale, deadline, w, o, dg);
    const bool retried = status < 0 && A.pass == 0 && A.single_shot < 0;   // goes to the overflow pass
    if (status < 0) {
        status = QEC_SHOT_CAPACITY;
        if (retried && T.tid() == 0) {
            const unsigned long long idx = atomicAdd(&A.queue[1], 1ull);
            A.overflow[idx] = (int)shot;
        }
        w = 0;
        o = 0;
    }
    if (dg && status != QEC_SHOT_OK && T.tid() < QEC_DIAG_FIELDS) dg[T.tid()] = 0;
    if constexpr (WIN) {
        // sliding window: nothing is committed by a failed shot
        if (status != QEC_SHOT_OK)
            for (int i = T.tid(); i < g.words; i += T.NT) A.carry[off + i] = 0u;
        if (T.tid() == 0) {
            if (status == QEC_SHOT_OK) A.cobs[shot] ^= o;
            else if (!retried) A.st_out[shot] = status;
        }
    } else if (T.tid() == 0) {
        A.w_out[shot] = w;
        A.obs_out[shot] = o;
        A.st_out[shot] = status;
        if (A.done && !retried) {
            // the results reach the host before the flag that publishes them
            __threadfence_system();
            asm volatile("st.release.sys.global.b32 [%0], %1;" :: "l"(A.done + shot), "r"(1) : "memory");
        }
    }
    T.sync();
}

// One team per warp (NW = 1, any block size that is a multiple of 32) or one
// team per block (NW > 1, blocks of exactly 32 NW threads).
template <bool WIN, int NW>
__global__ void __launch_bounds__(NW == 1 ? 128 : 32 * NW, NW == 1 ? QEC_MIN_BLOCKS : (NW == 4 ? 4 : 1))
batch_kernel(const __grid_constant__ BatchArgs a) {
    Team<NW> T;
    T.lane = threadIdx.x & 31;
    if constexpr (NW > 1) {
        __shared__ TeamShared tsh;
        T.sh = &tsh;
        T.tid_ = (int)threadIdx.x;
        T.warp_ = (int)(threadIdx.x >> 5);
        T.ph = 0;
    }
    const long long wid = NW == 1 ? (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) : (long long)blockIdx.x;
    Slab S;
    carve(a.slabs + wid * a.slab_bytes, a.caps, S);
    unsigned long long deadline = 0;
    if (a.watchdog_ns > 0) {
        unsigned long long t0 = T.tid() == 0 ? now_ns() : 0;
        deadline = T.bcast64(t0) + (unsigned long long)a.watchdog_ns;
    }
    if (a.single_shot >= 0) {
        if (wid == 0) decode_shot<WIN, NW>(a, S, a.single_shot, T, deadline);
        return;
    }
    unsigned long long *counter = a.queue + (a.pass == 0 ? 0 : 2);
    const long long limit = a.pass == 0 ? a.num_shots : (long long)min(a.queue[1], (unsigned long long)a.num_shots);
    for (long long it = 0; it < a.num_shots + 1; it++) {
        unsigned long long item = 0;
        if (T.tid() == 0) item = atomicAdd(counter, 1ull);
        item = T.bcast64(item);
        if ((long long)item >= limit) break;
        const long long shot = a.pass == 0 ? (a.order ? (long long)a.order[item] : (long long)item)
                                           : (long long)a.overflow[item];
        decode_shot<WIN, NW>(a, S, shot, T, deadline);
    }
}

struct GraphOrder {
    int g[QEC_MAX_GRAPHS_PER_BATCH];
};

__global__ void graph_count_kernel(const int *gid, long long n, int ng, int *gcnt) {
    __shared__ int local[QEC_MAX_GRAPHS_PER_BATCH];
    for (int i = threadIdx.x; i < QEC_MAX_GRAPHS_PER_BATCH; i += blockDim.x) local[i] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int g = gid[i];
        if (g < 0 || g >= ng) g = 0;
        atomicAdd(&local[g], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ng; i += blockDim.x)
        if (local[i]) atomicAdd(&gcnt[i], local[i]);
}

__global__ void graph_scan_kernel(int *gcnt, int ng, GraphOrder go) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int acc = 0;
    for (int k = 0; k < ng; k++) {
        const int g = go.g[k];
        gcnt[32 + g] = acc;
        acc += gcnt[g];
    }
}

__global__ void graph_scatter_kernel(const int *gid, long long n, int ng, int *gcnt, int *order) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int g = gid[i];
        if (g < 0 || g >= ng) g = 0;
        const int pos = atomicAdd(&gcnt[32 + g], 1);
        order[pos] = (int)i;
    }
}

}  // namespace

cudaError_t launch_graph_sort(const int *graph_of_shot, long long n, int ng, const int *gorder, int *gcnt,
                              int *order, cudaStream_t s) {
    GraphOrder go;
    for (int k = 0; k < QEC_MAX_GRAPHS_PER_BATCH; k++) go.g[k] = k < ng ? gorder[k] : 0;
    cudaError_t e = cudaMemsetAsync(gcnt, 0, 64 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    graph_count_kernel<<<blocks, 256, 0, s>>>(graph_of_shot, n, ng, gcnt);
    graph_scan_kernel<<<1, 32, 0, s>>>(gcnt, ng, go);
    graph_scatter_kernel<<<blocks, 256, 0, s>>>(graph_of_shot, n, ng, gcnt, order);
    return cudaGetLastError();
}

long long slab_bytes_for(const SlabCaps &c) {
    Slab S;
    long long b = carve(reinterpret_cast<char *>(0), c, S);
    return (b + 255) & ~255LL;
}

SlabCaps caps_for_kcap(int kcap, int table_factor) {
    auto p2 = [](long long x) { long long r = 1; while (r < x) r <<= 1; return (int)r; };
    const long long f = table_factor < 1 ? 1 : table_factor;
    SlabCaps c;
    c.kc = kcap;
    c.hc = p2(64LL * f * kcap < 1024 ? 1024 : 64LL * f * kcap);
    c.ec = (int)(48 * f * kcap + 64);
    c.wc = (int)(48 * f * kcap + 64);
    c.phc = p2(16LL * f * f * kcap < 256 ? 256 : 16LL * f * f * kcap);   // dense shots: pairs grow ~ f^2
    c.nc = 2 * kcap + 16;
    c.wcap = QEC_STREAM_MAX_WORDS;   // rows up to 73,728 detectors; callers raise it for larger graphs
    c.cc = 24 * kcap + 64;
    return c;
}

cudaError_t launch_batch(const BatchArgs &a, int grid, int block, cudaStream_t s, int team) {
    if (a.carry) {
        if (team == TEAM_BIG) batch_kernel<true, TEAM_BIG><<<grid, 32 * TEAM_BIG, 0, s>>>(a);
        else batch_kernel<true, 1><<<grid, block, 0, s>>>(a);
    } else if (team == TEAM_BIG) {
        batch_kernel<false, TEAM_BIG><<<grid, 32 * TEAM_BIG, 0, s>>>(a);
    } else if (team == TEAM_MID) {
        batch_kernel<false, TEAM_MID><<<grid, 32 * TEAM_MID, 0, s>>>(a);
    } else {
        batch_kernel<false, 1><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int max_block_threads() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, batch_kernel<false, 1>) != cudaSuccess) return 32;
    return fa.maxThreadsPerBlock > 0 ? fa.maxThreadsPerBlock : 32;
}

int occupancy_blocks(int block_threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<false, 1>, block_threads, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

int team_occupancy_blocks(int team) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (team == TEAM_BIG) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<false, TEAM_BIG>, 32 * TEAM_BIG, 0);
    else if (team == TEAM_MID) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<false, TEAM_MID>, 32 * TEAM_MID, 0);
    if (e != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

namespace {

// 32 bits of `row` (of `words` words) starting at bit b (bits past the row are 0).
__device__ __forceinline__ unsigned bits32(const unsigned *row, long long words, long long b) {
    const long long w = b >> 5;
    const int sh = (int)(b & 31);
    const unsigned lo = w < words ? row[w] : 0u;
    const unsigned hi = (sh && w + 1 < words) ? row[w + 1] : 0u;
    return sh ? (lo >> sh) | (hi << (32 - sh)) : lo;
}

__device__ __forceinline__ unsigned low_mask(long long n) {   // bits [0, n) of a word, n clamped to [0, 32]
    return n <= 0 ? 0u : (n >= 32 ? ~0u : (1u << n) - 1u);
}

// One thread per (row, window word).
__global__ void window_assemble_kernel(const unsigned *src, long long src_words, long long bit_begin, int nbits,
                                       const unsigned *carry, long long carry_words, long long carry_begin,
                                       int carry_bits, unsigned *dst, long long dst_words, long long num_rows) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= num_rows * dst_words) return;
    const long long r = i / dst_words, w = i - r * dst_words;
    const long long b = w * 32;
    unsigned v = bits32(src + r * src_words, src_words, bit_begin + b) & low_mask(nbits - b);
    if (carry) v ^= bits32(carry + r * carry_words, carry_words, carry_begin + b) & low_mask(carry_bits - b);
    dst[i] = v;
}

}  // namespace

cudaError_t launch_window_assemble(const unsigned *src, long long src_words, long long bit_begin, int nbits,
                                   const unsigned *carry, long long carry_words, long long carry_begin,
                                   int carry_bits, unsigned *dst, long long dst_words, long long num_rows,
                                   cudaStream_t s) {
    const long long n = num_rows * dst_words;
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    const long long grid = (n + block - 1) / block;
    window_assemble_kernel<<<(unsigned)grid, block, 0, s>>>(src, src_words, bit_begin, nbits, carry, carry_words,
                                                             carry_begin, carry_bits, dst, dst_words, num_rows);
    return cudaGetLastError();
}

cudaError_t launch_reset_queue(unsigned long long *queue, cudaStream_t s) {
    return cudaMemsetAsync(queue, 0, 4 * sizeof(unsigned long long), s);
}

}  // namespace qec
