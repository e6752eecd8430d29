// trk_event.cu - persistent event-based kernel (sm_103a).
//
// Paper: Sec. 2.3 (event-based GPU transport: tracking operations run over a
// vector of histories, one operation at a time) on top of Alg. 2-10.
//
// GB300 design.  Each warp owns `slots` particle slots whose state lives in
// the caller's work buffer (one compact record per slot, 176 bytes for the
// CSG tracker, sized to stay in L2) and keeps its
// own queues of slot indices in shared memory: flight (distance_to_surface +
// move_within_cell + tally), cross (cross_surface + find_cell below),
// collide (change_direction), free.  A round runs refill, then flight over
// the whole flight queue, then cross and collide over theirs, all 32 lanes
// on one kind of operation, so the warp stays converged where the history
// kernel diverges.  Queue counts are warp-uniform registers advanced by
// ballot/popc; empty slots take new particles from one global counter.  No
// warp ever waits for another (only __syncwarp), and a round limit turns a
// runaway into TRK_E_TIMEOUT.
// Per-particle arithmetic is the history kernel's, so results are the same
// bit for bit.
#include <cstdint>

#include "trk.h"
#include "trk_device.cuh"
#include "trk_internal.h"
#include "trk_launch.h"

using namespace trk;
using namespace trk::dev;

namespace {

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

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t buf_bytes(long long T) { return 256 + align256(size_t(T) * size_t(rec_bytes<false>())); }

EvBuf make_buf(void* work, long long T) {
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

// Each warp owns `slots` particle slots and its own queues in shared memory;
// warps never synchronise with each other.
template <bool CSG, bool F32, int FLAGS>
__global__ void TRK_EV_BOUNDS k_event(const DevGeom g, const ParticlesView P, long long n, const RunP rp,
                                      const EvBuf B, int slots, unsigned long long max_rounds,
                                      unsigned long long* __restrict__ tally,
                                      unsigned long long* __restrict__ counters,
                                      unsigned long long* __restrict__ rec) {
    extern __shared__ QIdx smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    QIdx* base_q = smem + warp * EV_QUEUES * slots;
    QIdx* qfl = base_q;                  // NFC flight queues
    QIdx* qc = base_q + NFC * slots;     // collide (at refill: failed births)
    QIdx* qf = base_q + (NFC + 1) * slots;
    QIdx* qx = base_q + (NFC + 2) * slots;   // MAXL cross queues, one per crossing level
    const int slot0 = (blockIdx.x * (EV_BLOCK / 32) + warp) * slots;
    Counts cnt;
#pragma unroll
    for (int k = 0; k < NCOUNT; ++k) cnt.k[k] = 0;
    for (int k = lane; k < slots; k += 32) qf[k] = QIdx(k);
    int n_fl[NFC];
#pragma unroll
    for (int c = 0; c < NFC; ++c) n_fl[c] = 0;
    int n_free = slots;
    bool exhausted = false;
    __syncwarp();
    for (unsigned long long round = 0;; ++round) {
        // ---- refill free slots with new particles --------------------------
        // in batches of at least a warp's width (birth runs the universe
        // searches from the root, whose lanes diverge least when the batch
        // is full), unless the flight queues are running low
        int n_live = 0;
#pragma unroll
        for (int q = 0; q < NFC; ++q) n_live += n_fl[q];
        int got = 0;
        unsigned long long first = 0;
        if (!exhausted && n_free > 0 && (n_free >= TRK_EV_REFILL_MIN || n_live < 32)) {
            if (lane == 0) first = atomicAdd(B.ctr, (unsigned long long)n_free);
            first = __shfl_sync(0xffffffffu, first, 0);
            long long avail = (long long)n - (long long)first;
            if (avail <= 0) { avail = 0; exhausted = true; }
            if (avail >= n_free) got = n_free;
            else { got = int(avail); exhausted = true; }
        }
        int n_park = 0;
        for (int b = 0; b < got; b += 32) {
            const int k = b + lane;
            bool ok = false;
            int slot = 0, cls = 0;
            if (k < got) {
                slot = slot0 + qf[n_free - got + k];
                const long long pidx = (long long)first + k;
                Ctx c;
                c.pid = uint32_t(rp.first_id + uint64_t(pidx));
                c.event = 0; c.nseg = 0; c.path = 0.0; c.hash = FNV0; c.status = 0;
                const int pst = P.status[pidx];
                if (pst != 0) {
                    c.status = pst;
                    cnt.k[TRK_K_SOURCE]++;
                } else {
                    St s;
                    load_birth(g, P, pidx, s);
                    if (find_from<CSG>(g, s, 0) != 0) {
                        c.status = TRK_E_LOST;
                        cnt.k[TRK_K_LOST]++;
                    } else {
                        unsigned char* r = rec_at<CSG>(B, slot);
                        cls = flight_class<CSG>(g, s);
                        D2(r, R_XY) = make_double2(s.x, s.y);
                        D2(r, R_ZT) = make_double2(s.z, s.tau);
                        store_dir(r, s);
                        store_levels<CSG>(r, s, cls);
                        store_ctx<FLAGS>(r, int(pidx), c, 0);
                        ok = true;
                    }
                }
                if (!ok) finish<FLAGS>(pidx, c, rec);
            }
#pragma unroll
            for (int q = 0; q < NFC; ++q) wpush(ok && cls == q, slot - slot0, qfl + q * slots, n_fl[q]);
            wpush(k < got && !ok, slot - slot0, qc, n_park);
        }
        __syncwarp();
        n_free -= got;
        for (int b = 0; b < n_park; b += 32) {
            const int k = b + lane;
            wpush(k < n_park, k < n_park ? qc[k] : 0, qf, n_free);
        }
        __syncwarp();
        int n_fly = 0;
#pragma unroll
        for (int q = 0; q < NFC; ++q) n_fly += n_fl[q];
        if (n_fly == 0 && exhausted) break;
        if (round >= max_rounds) {
            if (lane == 0) kernel_status(counters, TRK_E_TIMEOUT);
            break;
        }
        // ---- flight: distance_to_surface, tally, move ----------------------
        // the class queues are walked as one concatenated list
        int n_cross[MAXL], n_coll = 0;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) n_cross[l] = 0;
        for (int b = 0; b < n_fly; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0, hl = -1;
            if (k < n_fly) {
                int q = 0, kk = k;
#pragma unroll
                for (int c = 0; c < NFC - 1; ++c)
                    if (q == c && kk >= n_fl[c]) { kk -= n_fl[c]; q = c + 1; }
                slot = slot0 + qfl[q * slots + kk];
                unsigned char* r = rec_at<CSG>(B, slot);
                St s;
                const double2 xy = D2(r, R_XY), zt = D2(r, R_ZT);
                s.x = xy.x; s.y = xy.y; s.z = zt.x; s.tau = zt.y;
                load_dir(r, s);
                load_levels<CSG>(g, r, s);
                Ctx c;
                int hpack;
                const int pidx = load_ctx<FLAGS>(r, c, hpack, rp);
                Hit h;
                a = step_fly<CSG, F32, FLAGS>(g, s, h, c, rp, tally, cnt, nullptr, nullptr, 0);
                if (a == A_DONE) {
                    finish<FLAGS>(pidx, c, rec);
                } else {
                    D2(r, R_XY) = make_double2(s.x, s.y);
                    D2(r, R_ZT) = make_double2(s.z, s.tau);
                    if (a == A_CROSS) {
                        hl = h.level;
                        store_ctx<FLAGS>(r, pidx, c, pack_hit(h));
                        I4(r, R_HT) = make_int4(h.surf, h.entry, 0, 0);
                    } else {
                        store_ctx<FLAGS>(r, pidx, c, hpack);
                    }
                }
            }
            const bool live = k < n_fly;
            // crossings are queued by level, so each pass runs one code path
            // (array index step, universe search, pin cell test)
#pragma unroll
            for (int l = 0; l < MAXL; ++l) wpush(live && hl == l, slot - slot0, qx + l * slots, n_cross[l]);
            wpush(live && a == A_COLLIDE, slot - slot0, qc, n_coll);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NFC; ++q) n_fl[q] = 0;
        // ---- cross_surface, then change_direction ---------------------------
#pragma unroll 1
        for (int lq = 0; lq < MAXL; ++lq)
        for (int b = 0; b < n_cross[lq]; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0, cls = 0;
            if (k < n_cross[lq]) {
                slot = slot0 + qx[lq * slots + k];
                unsigned char* r = rec_at<CSG>(B, slot);
                St s;
                const double2 xy = D2(r, R_XY), zt = D2(r, R_ZT);
                s.x = xy.x; s.y = xy.y; s.z = zt.x; s.tau = zt.y;
                load_dir(r, s);
                load_levels<CSG>(g, r, s);
                Ctx c;
                int hpack;
                const int pidx = load_ctx<FLAGS>(r, c, hpack, rp);
                Hit h;
                unpack_hit(hpack, h);
                const int4 ht = I4(r, R_HT);
                h.surf = ht.x; h.entry = ht.y; h.d = 0.0;
                const unsigned refl0 = cnt.k[TRK_K_REFLECTIONS];
                a = step_cross<CSG>(g, s, h, c, rp, cnt);
                if (a == A_DONE) {
                    finish<FLAGS>(pidx, c, rec);
                } else {
                    cls = flight_class<CSG>(g, s);
                    store_levels<CSG>(r, s, cls);
                    if (cnt.k[TRK_K_REFLECTIONS] != refl0) store_dir(r, s);
                }
            }
            const bool live = k < n_cross[lq];
#pragma unroll
            for (int q = 0; q < NFC; ++q) wpush(live && a == A_FLY && cls == q, slot - slot0, qfl + q * slots, n_fl[q]);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
        }
        for (int b = 0; b < n_coll; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0, cls = 0;
            if (k < n_coll) {
                slot = slot0 + qc[k];
                unsigned char* r = rec_at<CSG>(B, slot);
                St s;
                Ctx c;
                int hpack;
                const int pidx = load_ctx<FLAGS>(r, c, hpack, rp);
                a = step_collide(g, s, c, rp, cnt);
                if (a == A_DONE) {
                    finish<FLAGS>(pidx, c, rec);
                } else {
                    store_dir(r, s);
                    const double z = D2(r, R_ZT).x;
                    D2(r, R_ZT) = make_double2(z, s.tau);
                    const int4 lv = I4(r, R_LV);
                    cls = lv.x >> 16;
                    I4(r, R_LV) = make_int4(lv.x, -1, -1, lv.w);
                    store_ctx<FLAGS>(r, pidx, c, hpack);
                }
            }
            const bool live = k < n_coll;
#pragma unroll
            for (int q = 0; q < NFC; ++q) wpush(live && a == A_FLY && cls == q, slot - slot0, qfl + q * slots, n_fl[q]);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
        }
        __syncwarp();
    }
    flush_counts(cnt, counters);
}

}  // namespace

namespace trk {

constexpr int EV_WARPS = EV_BLOCK / 32;

// Resident CTAs per SM: the register budget's minimum (TRK_EV_MINB), capped
// by shared memory.  Deterministic, so the work-buffer size a caller queries
// always matches the launch.
int event_grid(int slots) {
    int dev = 0, sms = 152, smem_sm = 228 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    const size_t smem = size_t(EV_QUEUES) * slots * EV_WARPS * sizeof(QIdx);
    const int by_smem = int(size_t(smem_sm) / (smem + 1024));
    int per_sm = TRK_EV_MINB > 0 ? TRK_EV_MINB : 1;
    if (per_sm > by_smem) per_sm = by_smem;
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

size_t event_work_bytes(int slots, int grid) { return buf_bytes((long long)slots * EV_WARPS * grid); }

trk_status launch_event(trk_geom_t g, const ParticlesView& P, long long n, const RunP& rp, bool csg, bool f32,
                        int flags, unsigned long long* tally, unsigned long long* cnt, unsigned long long* rec,
                        void* work, size_t work_bytes, int slots, int grid, int max_rounds_opt, cudaStream_t s) {
    const long long T = (long long)slots * EV_WARPS * grid;
    if (work_bytes < buf_bytes(T) || !work)
        return trk_status(set_error(TRK_E_NOMEM, "run_histories (event): work buffer needs %zu bytes", buf_bytes(T)));
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return trk_status(set_error(TRK_E_INVALID, "run_histories (event): work buffer must be 256-byte aligned"));
    const EvBuf B = make_buf(work, T);
    cudaError_t e = cudaMemsetAsync(B.ctr, 0, 8, s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_histories (event): %s", cudaGetErrorString(e)));
    const size_t smem = size_t(EV_QUEUES) * slots * EV_WARPS * sizeof(QIdx);
    // a particle needs at most max_segments + 1 flight rounds; a warp holds
    // `slots` particles at a time and refills every round
    const unsigned long long per_warp = (unsigned long long)(n / (T / slots) + slots + 1);
    unsigned long long max_rounds = (rp.max_segments + 2ULL) * (per_warp / slots + 2ULL) * 4ULL;
    if (max_rounds_opt > 0) max_rounds = (unsigned long long)max_rounds_opt;
#define TRK_EV(C, F32V, F)                                                                                   \
    do {                                                                                                     \
        auto k = k_event<C, F32V, F>;                                                                        \
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); \
        k<<<grid, EV_BLOCK, smem, s>>>(g->dg, P, n, rp, B, slots, max_rounds, tally, cnt, rec);             \
    } while (0)
    if (f32) {
#ifndef TRK_EXACT
        if (csg) {
            if (flags & F_REC) TRK_EV(true, true, F_REC);
            else TRK_EV(true, true, 0);
        } else {
            if (flags & F_REC) TRK_EV(false, true, F_REC);
            else TRK_EV(false, true, 0);
        }
#endif
    } else if (csg) {
        switch (flags) {
            case 0: TRK_EV(true, false, 0); break;
            case F_REC: TRK_EV(true, false, F_REC); break;
            case F_CUT: TRK_EV(true, false, F_CUT); break;
            default: TRK_EV(true, false, F_REC | F_CUT); break;
        }
    } else {
        switch (flags) {
            case 0: TRK_EV(false, false, 0); break;
            case F_REC: TRK_EV(false, false, F_REC); break;
            case F_CUT: TRK_EV(false, false, F_CUT); break;
            default: TRK_EV(false, false, F_REC | F_CUT); break;
        }
    }
#undef TRK_EV
    e = cudaGetLastError();
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_histories (event): %s", cudaGetErrorString(e)));
    return TRK_OK;
}

}  // namespace trk
