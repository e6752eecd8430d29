// trk_event.cuh - the event kernels' slot records, warp queues and launch
// shape, shared by the single-geometry event kernel (trk_event.cu) and the
// batched one (batch.cu).  Not part of the ABI.
#pragma once
#include <cstdint>

#include "trk.h"
#include "trk_device.cuh"
#include "trk_internal.h"

namespace trk {
namespace ev {

using namespace trk::dev;

constexpr int EV_BLOCK = 256;
// Flight queue entries carry the class of the particle's leaf cell (cells
// whose distance code takes the same path: no curved surface, one cylinder
// from inside, one from outside, other) above the slot index; every
// sort_interval rounds (trk_run_opts) the warp reorders its flight queue by
// that class before the flight pass, so a flight batch's lanes mostly run
// the same branches.
constexpr int QSLOT_BITS = 12;
constexpr unsigned QSLOT_MASK = (1u << QSLOT_BITS) - 1u;
constexpr int NCLASS = 4;
// Queue entries are slot indices within the warp's own range (< 512) and,
// in the flight queue, the class bits above them: 16 bits each, half the
// shared memory of 32-bit entries, which the L1 cache gets.
using QIdx = unsigned short;
// Free slots a warp collects before it refills them (see the refill step):
// the single-geometry event kernel refills 128 at a time (measured 1.3-1.8%
// ahead of 32 on the 15 x 15 and hex cores), the batched one 32 (its chunks
// are short).
#ifndef TRK_EV_REFILL_MIN
#define TRK_EV_REFILL_MIN 128
#endif
#ifndef TRK_BEV_REFILL_MIN
#define TRK_BEV_REFILL_MIN 32
#endif
constexpr int EV_QUEUES = 4 + MAXL;   // flight, collide, free, FP64 redo, cross per level

// Minimum resident CTAs per SM the register allocation must allow (0: let
// the compiler choose).  Two CTAs (16 warps, 128 registers a thread) hide
// more latency than one CTA with the whole state in registers; the spills
// this costs are a few dozen bytes in the rect and FP32 variants.
#ifndef TRK_EV_MINB
#define TRK_EV_MINB 2
#endif
#if TRK_EV_MINB > 0
#define TRK_EV_BOUNDS __launch_bounds__(EV_BLOCK, TRK_EV_MINB)
#else
#define TRK_EV_BOUNDS __launch_bounds__(EV_BLOCK)
#endif

// Slot record: one 16-byte-aligned record per slot, read and written in
// 16-byte chunks (a lane's fields share sectors whatever order the queues
// put the slots in).  Only what a history needs between operations is kept,
// packed so that the records of all slots stay small next to the L2 cache:
//    0  x, y                16  z, tau
//   32  u, v                48  w, 1/u
//   64  1/v, 1/w            80  per level the cell (rect levels: i | j << 10 | k << 20)
//   96  particle index, event, segments, misc
//  112  on-surface surface, hit reference, universes of levels 0|1, 2|3 (16 bits each)
//  128  record hash, path length (only with records or a path cutoff)
// misc: hit level, side, dim, sign (9 bits) | levels << 9 | (on-surface level
// + 1) << 12 | flight class << 15 | material << 17.  The hit reference is the
// crossed entry of the cell's surface list, or for a rect array face its
// negative face code (the surface follows from either).  Translations and
// instance offsets are reloaded from the geometry tables.
static_assert(MAXL == 4, "the slot record keeps one int4 of cells");
constexpr int R_XY = 0, R_ZT = 16, R_UV = 32, R_WI = 48, R_II = 64, R_LC = 80, R_CT = 96, R_SU = 112, R_HP = 128;
// Limits of the packed fields (checked on the host before an event launch).
constexpr int REC_MAX_DIM = 1024;        // rect array elements per axis
constexpr int REC_MAX_UNIV = 1 << 16;    // universes
constexpr int REC_MAX_MAT = 1 << 15;     // materials

template <int FLAGS>
__host__ __device__ constexpr int rec_bytes() { return (FLAGS & (F_REC | F_CUT)) ? 144 : 128; }
constexpr int REC_BYTES_MAX = 144;

struct EvBuf {
    unsigned char* rec;
    unsigned long long* ctr;    // [0] next particle index
    long long T;                // total slots
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline size_t buf_bytes(long long T) { return 256 + align256(size_t(T) * size_t(REC_BYTES_MAX)); }

inline EvBuf make_buf(void* work, long long T) {
    unsigned char* b = static_cast<unsigned char*>(work);
    EvBuf e;
    e.ctr = reinterpret_cast<unsigned long long*>(b);
    e.rec = b + 256;
    e.T = T;
    return e;
}

template <int FLAGS>
__device__ __forceinline__ unsigned char* rec_at(const EvBuf& B, int s) {
    return B.rec + (size_t)s * rec_bytes<FLAGS>();
}
__device__ __forceinline__ double2& D2(unsigned char* r, int off) { return *reinterpret_cast<double2*>(r + off); }
__device__ __forceinline__ int4& I4(unsigned char* r, int off) { return *reinterpret_cast<int4*>(r + off); }
__device__ __forceinline__ longlong2& L2(unsigned char* r, int off) { return *reinterpret_cast<longlong2*>(r + off); }

__device__ __forceinline__ int pack_hit(const Hit& h) {
    return (h.level + 1) | ((h.side + 1) << 3) | ((h.dim + 1) << 5) | ((h.dsign + 1) << 7);
}
__device__ __forceinline__ void unpack_hit(int p, Hit& h) {
    h.level = (p & 7) - 1; h.side = ((p >> 3) & 3) - 1; h.dim = ((p >> 5) & 3) - 1; h.dsign = ((p >> 7) & 3) - 1;
}
__device__ __forceinline__ int hit_ref(const Hit& h) { return h.surf < 0 ? h.surf : h.entry; }
__device__ __forceinline__ void hit_from_ref(const DevGeom& g, int ref, Hit& h) {
    if (ref < 0) { h.surf = ref; h.entry = -1; }
    else { h.entry = ref; h.surf = cs_surface(__ldg(g.cs + ref)); }
}

__device__ __forceinline__ unsigned make_misc(int hpack, const St& st, int cls) {
    return unsigned(hpack) | (unsigned(st.nlev) << 9) | (unsigned(st.on_lev + 1) << 12) | (unsigned(cls) << 15) |
           (unsigned(st.mat) << 17);
}
__device__ __forceinline__ int misc_hpack(unsigned m) { return int(m & 511u); }
__device__ __forceinline__ int misc_cls(unsigned m) { return int((m >> 15) & 3u); }
__device__ __forceinline__ int misc_mat(unsigned m) { return int(m >> 17); }
// misc with the hit replaced
__device__ __forceinline__ unsigned misc_with_hit(unsigned m, int hpack) { return (m & ~511u) | unsigned(hpack); }
// misc with the on-surface level cleared (after a collision)
__device__ __forceinline__ unsigned misc_off_surface(unsigned m) { return m & ~(7u << 12); }

// Translation and instance offset of every occupied level, from the tables
// the find and cross steps take them from (the same values, bit for bit).
template <bool CSG>
__device__ __forceinline__ void reload_frames(const DevGeom& g, St& st) {
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        Lv& L = st.lv[l];
        if (l >= st.nlev) { L.tx = L.ty = L.tz = 0.0; L.off = 0; continue; }
        const int lat = CSG ? -1 : __ldg(g.u_info + L.u).w;
        if (lat >= 0) {
            const int4 of = __ldg(g.l_off + lat);
            const int4 dm = __ldg(g.l_dim + lat);
            L.cell = L.i + dm.x * (L.j + dm.y * L.k);
            L.off = __ldg(g.l_eoff + of.w + L.cell);
            L.tx = __ldg(g.l_ctr + of.x + L.i);
            L.ty = __ldg(g.l_ctr + of.y + L.j);
            L.tz = __ldg(g.l_ctr + of.z + L.k);
        } else {
            L.off = __ldg(g.c_off + L.cell);
            L.tx = __ldg(g.c_tr + 3 * L.cell);
            L.ty = __ldg(g.c_tr + 3 * L.cell + 1);
            L.tz = __ldg(g.c_tr + 3 * L.cell + 2);
        }
    }
}

// Level stack from the cells chunk, the misc word and the universes chunk.
// A rect level's cell word holds i, j, k; its element index is rebuilt.
template <bool CSG>
__device__ __forceinline__ void load_levels(const DevGeom& g, unsigned char* r, St& st, unsigned misc, const int4& su) {
    st.nlev = int((misc >> 9) & 7u);
    st.on_lev = int((misc >> 12) & 7u) - 1;
    st.mat = misc_mat(misc);
    st.on_surf = su.x;
    const int4 lc = I4(r, R_LC);
    const int c4[4] = {lc.x, lc.y, lc.z, lc.w};
    const int u4[4] = {su.z & 0xffff, int(unsigned(su.z) >> 16), su.w & 0xffff, int(unsigned(su.w) >> 16)};
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        st.lv[l].u = u4[l];
        st.lv[l].cell = c4[l];
        st.lv[l].i = st.lv[l].j = st.lv[l].k = 0;
        if (!CSG) {
            st.lv[l].i = c4[l] & 1023;
            st.lv[l].j = (c4[l] >> 10) & 1023;
            st.lv[l].k = (c4[l] >> 20) & 1023;
        }
    }
    reload_frames<CSG>(g, st);
}

// Flight class of the particle's leaf cell (a rect-array leaf is class 0).
template <bool CSG>
__device__ __forceinline__ int flight_class(const DevGeom& g, const St& st) {
    const Lv L = lv_get(st, st.nlev - 1);
    if (!CSG && __ldg(g.u_info + L.u).w >= 0) return 0;
    const int c = __ldg(g.c_fcls + L.cell);
    return c < NCLASS ? c : NCLASS - 1;
}

// Stable counting sort of a warp's queue list[0..n) by the class bits of its
// entries into out[0..n) (all 32 lanes call; ballots keep lane order).
__device__ __forceinline__ void sort_by_class(const QIdx* list, int n, QIdx* out) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int off[NCLASS];
#pragma unroll
    for (int c = 0; c < NCLASS; ++c) off[c] = 0;
    for (int b = 0; b < n; b += 32) {
        const int k = b + lane;
        const int c = k < n ? int(unsigned(list[k]) >> QSLOT_BITS) : NCLASS;
#pragma unroll
        for (int q = 0; q < NCLASS; ++q) off[q] += __popc(__ballot_sync(0xffffffffu, c == q));
    }
    int start = 0;
#pragma unroll
    for (int q = 0; q < NCLASS; ++q) { const int t = off[q]; off[q] = start; start += t; }
    for (int b = 0; b < n; b += 32) {
        const int k = b + lane;
        const QIdx e = k < n ? list[k] : QIdx(0);
        const int c = k < n ? int(unsigned(e) >> QSLOT_BITS) : NCLASS;
#pragma unroll
        for (int q = 0; q < NCLASS; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, c == q);
            if (c == q) out[off[q] + __popc(m & below)] = e;
            off[q] += __popc(m);
        }
    }
    __syncwarp();
}

// The cells chunk and the universes word (on-surface surface, hit reference,
// universes); rect levels store i, j, k in the cell word.
template <bool CSG>
__device__ __forceinline__ int4 store_levels(const DevGeom& g, unsigned char* r, const St& st, int href) {
    int c4[4];
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        c4[l] = st.lv[l].cell;
        if (!CSG && l < st.nlev && __ldg(g.u_info + st.lv[l].u).w >= 0)
            c4[l] = st.lv[l].i | (st.lv[l].j << 10) | (st.lv[l].k << 20);
    }
    I4(r, R_LC) = make_int4(c4[0], c4[1], c4[2], c4[3]);
    const int4 su = make_int4(st.on_surf, href, (st.lv[0].u & 0xffff) | (st.lv[1].u << 16),
                              (st.lv[2].u & 0xffff) | (st.lv[3].u << 16));
    I4(r, R_SU) = su;
    return su;
}

__device__ __forceinline__ void load_dir(unsigned char* r, St& st) {
    const double2 uv = D2(r, R_UV), wi = D2(r, R_WI), ii = D2(r, R_II);
    st.d.u = uv.x; st.d.v = uv.y; st.d.w = wi.x; st.d.iu = wi.y; st.d.iv = ii.x; st.d.iw = ii.y;
}

__device__ __forceinline__ void store_dir(unsigned char* r, const St& st) {
    D2(r, R_UV) = make_double2(st.d.u, st.d.v);
    D2(r, R_WI) = make_double2(st.d.w, st.d.iu);
    D2(r, R_II) = make_double2(st.d.iv, st.d.iw);
}

// Context of a live history (status is 0 while it lives) from the ctx
// chunk; returns the particle's index in this launch and sets misc.
template <int FLAGS>
__device__ __forceinline__ int load_ctx(unsigned char* r, Ctx& c, unsigned& misc, const RunP& rp) {
    const int4 ct = I4(r, R_CT);
    c.pid = uint32_t(rp.first_id + uint64_t(uint32_t(ct.x)));
    c.event = uint32_t(ct.y);
    c.nseg = (long long)(uint32_t)ct.z;
    misc = unsigned(ct.w);
    c.status = 0;
    c.hash = 0; c.path = 0.0;
    if (FLAGS & (F_REC | F_CUT)) {
        const longlong2 hp = L2(r, R_HP);
        c.hash = (uint64_t)hp.x;
        c.path = __longlong_as_double(hp.y);
    }
    return ct.x;
}

template <int FLAGS>
__device__ __forceinline__ void store_ctx(unsigned char* r, int pidx, const Ctx& c, unsigned misc) {
    I4(r, R_CT) = make_int4(pidx, int(c.event), int(uint32_t(c.nseg)), int(misc));
    if (FLAGS & (F_REC | F_CUT)) L2(r, R_HP) = make_longlong2((long long)c.hash, __double_as_longlong(c.path));
}

// Entries of a queue a pass runs: whole 32-lane batches only, the tail
// staying queued for a later round, unless the round drains (the warp's
// source is exhausted, or no queue holds a full batch), when everything
// runs.  A pass then spends a warp-wide step on a batch with a few live
// lanes only where nothing else is left to run, and every round advances.
__device__ __forceinline__ int batch_run(int n, bool drain) { return drain ? n : (n & ~31); }

// Moves the n - done entries left after a pass (fewer than 32, with done a
// multiple of 32, or none) to the front of the queue; all 32 lanes call.
__device__ __forceinline__ void carry_tail(QIdx* q, int done, int& n) {
    const int lane = threadIdx.x & 31;
    const int rem = n - done;
    if (done > 0 && rem > 0) {
        // rem < 32 <= done: the source and destination ranges are disjoint
        if (lane < rem) q[lane] = q[done + lane];
    }
    n = rem;
    __syncwarp();
}

// Warp-level append of `v` to `list` when `flag` (all 32 lanes call);
// `count` is warp-uniform and advanced in every lane.
__device__ __forceinline__ void wpush(bool flag, int v, QIdx* list, int& count) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31;
    if (flag) list[count + __popc(m & ((1u << lane) - 1u))] = QIdx(v);
    count += __popc(m);
}

template <int FLAGS>
__device__ __forceinline__ void finish(long long pidx, const Ctx& c, unsigned long long* rec) {
    if (FLAGS & F_REC) {
        rec[2 * pidx] = c.hash;
        rec[2 * pidx + 1] = (uint64_t(c.nseg) << 32) | uint32_t(c.status);
    }
}

// Segment log (F_TRACE): entries past a finished history's last segment
// read instance -1, length 0.
template <int FLAGS>
__device__ __forceinline__ void trace_tail(long long pidx, const Ctx& c, const RunP& rp) {
    if (FLAGS & F_TRACE) {
        for (long long k = c.nseg; k < rp.trace_cap; ++k) {
            rp.tr_inst[pidx * rp.trace_cap + k] = -1;
            rp.tr_len[pidx * rp.trace_cap + k] = 0.0;
        }
    }
}

}  // namespace ev
}  // namespace trk
