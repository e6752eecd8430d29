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
// Flight queues by the class of the particle's leaf cell (cells whose
// distance code takes the same path: no curved surface, one cylinder from
// inside, one from outside, other), so a flight batch's lanes mostly run the
// same branches; the classes are concatenated in one pass, so a partial batch
// occurs only once per flight phase.  Measured on the three-level core, the
// sorting does not pay for its extra queue traffic (4 classes: -2 to -5%), so
// the default is one class.
#ifndef TRK_EV_NFC
#define TRK_EV_NFC 1
#endif
constexpr int NFC = TRK_EV_NFC;
// Free slots a warp collects before it refills them (see the refill step).
#ifndef TRK_EV_REFILL_MIN
#define TRK_EV_REFILL_MIN 32
#endif
constexpr int EV_QUEUES = NFC + 2 + MAXL;   // flight by class, collide, free, cross per level

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
// put the slots in).  Only what a history needs between operations is kept:
// per level the universe and cell (rect levels also i, j, k); translations
// and instance offsets are reloaded from the geometry tables.
static_assert(MAXL == 4, "the slot record keeps one int4 per level field");
constexpr int R_XY = 0,     // x, y
              R_ZT = 16,    // z, tau
              R_UV = 32,    // u, v
              R_WI = 48,    // w, 1/u
              R_II = 64,    // 1/v, 1/w
              R_HP = 80,    // record hash, path length (only with records / path cutoff)
              R_LV = 96,    // nlev | flight class << 16, on_lev, on_surf, mat
              R_CT = 112,   // particle index, event, segments, packed hit (level, side, dim, sign)
              R_HT = 128,   // hit surface, hit entry
              R_LU = 144,   // universe per level
              R_LC = 160,   // cell (rect: element) per level
              R_LI = 176, R_LJ = 192, R_LK = 208;   // rect levels: i, j, k
template <bool CSG>
__host__ __device__ constexpr int rec_bytes() { return CSG ? 176 : 224; }

struct EvBuf {
    unsigned char* rec;
    unsigned long long* ctr;    // [0] next particle index
    long long T;                // total slots
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline size_t buf_bytes(long long T) { return 256 + align256(size_t(T) * size_t(rec_bytes<false>())); }

inline EvBuf make_buf(void* work, long long T) {
    unsigned char* b = static_cast<unsigned char*>(work);
    EvBuf e;
    e.ctr = reinterpret_cast<unsigned long long*>(b);
    e.rec = b + 256;
    e.T = T;
    return e;
}

template <bool CSG>
__device__ __forceinline__ unsigned char* rec_at(const EvBuf& B, int s) {
    return B.rec + (size_t)s * rec_bytes<CSG>();
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

template <bool CSG>
__device__ __forceinline__ void load_levels(const DevGeom& g, unsigned char* r, St& st) {
    const int4 lv = I4(r, R_LV);
    st.nlev = lv.x & 0xffff; st.on_lev = lv.y; st.on_surf = lv.z; st.mat = lv.w;
    const int4 lu = I4(r, R_LU), lc = I4(r, R_LC);
    const int u4[4] = {lu.x, lu.y, lu.z, lu.w}, c4[4] = {lc.x, lc.y, lc.z, lc.w};
#pragma unroll
    for (int l = 0; l < MAXL; ++l) { st.lv[l].u = u4[l]; st.lv[l].cell = c4[l]; st.lv[l].i = st.lv[l].j = st.lv[l].k = 0; }
    if (!CSG) {
        const int4 li = I4(r, R_LI), lj = I4(r, R_LJ), lk = I4(r, R_LK);
        const int i4[4] = {li.x, li.y, li.z, li.w}, j4[4] = {lj.x, lj.y, lj.z, lj.w}, k4[4] = {lk.x, lk.y, lk.z, lk.w};
#pragma unroll
        for (int l = 0; l < MAXL; ++l) { st.lv[l].i = i4[l]; st.lv[l].j = j4[l]; st.lv[l].k = k4[l]; }
    }
    reload_frames<CSG>(g, st);
}

// Flight class of the particle's leaf cell (a rect-array leaf is class 0).
template <bool CSG>
__device__ __forceinline__ int flight_class(const DevGeom& g, const St& st) {
    if (NFC == 1) return 0;
    const Lv L = lv_get(st, st.nlev - 1);
    if (!CSG && __ldg(g.u_info + L.u).w >= 0) return 0;
    const int c = __ldg(g.c_fcls + L.cell);
    return c < NFC ? c : NFC - 1;
}

// The level fields; the flight class rides in the upper half of nlev's word.
template <bool CSG>
__device__ __forceinline__ void store_levels(unsigned char* r, const St& st, int cls) {
    I4(r, R_LV) = make_int4(st.nlev | (cls << 16), st.on_lev, st.on_surf, st.mat);
    I4(r, R_LU) = make_int4(st.lv[0].u, st.lv[1].u, st.lv[2].u, st.lv[3].u);
    I4(r, R_LC) = make_int4(st.lv[0].cell, st.lv[1].cell, st.lv[2].cell, st.lv[3].cell);
    if (!CSG) {
        I4(r, R_LI) = make_int4(st.lv[0].i, st.lv[1].i, st.lv[2].i, st.lv[3].i);
        I4(r, R_LJ) = make_int4(st.lv[0].j, st.lv[1].j, st.lv[2].j, st.lv[3].j);
        I4(r, R_LK) = make_int4(st.lv[0].k, st.lv[1].k, st.lv[2].k, st.lv[3].k);
    }
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

// Context of a live history (status is 0 while it lives).  Returns the
// particle's index in this launch.
template <int FLAGS>
__device__ __forceinline__ int load_ctx(unsigned char* r, Ctx& c, int& hpack, const RunP& rp) {
    const int4 ct = I4(r, R_CT);
    c.pid = uint32_t(rp.first_id + uint64_t(uint32_t(ct.x)));
    c.event = uint32_t(ct.y);
    c.nseg = (long long)(uint32_t)ct.z;
    hpack = ct.w;
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
__device__ __forceinline__ void store_ctx(unsigned char* r, int pidx, const Ctx& c, int hpack) {
    I4(r, R_CT) = make_int4(pidx, int(c.event), int(uint32_t(c.nseg)), hpack);
    if (FLAGS & (F_REC | F_CUT)) L2(r, R_HP) = make_longlong2((long long)c.hash, __double_as_longlong(c.path));
}

// Warp-level append of `v` to `list` when `flag` (all 32 lanes call);
// `count` is warp-uniform and advanced in every lane.
// Queue entries are slot indices within the warp's own range (< 512), 16 bits
// each: half the shared memory of 32-bit entries, which the L1 cache gets.
using QIdx = unsigned short;

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

}  // namespace ev
}  // namespace trk
