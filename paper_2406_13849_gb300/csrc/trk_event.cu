// trk_event.cu - persistent event-based kernel (sm_103a).
//
// Paper: Sec. 2.3 (event-based GPU transport: tracking operations run over a
// vector of histories, one operation at a time) on top of Alg. 2-10.
//
// GB300 design.  Each warp owns `slots` particle slots whose state lives in
// the caller's work buffer (structure of arrays, L2-resident) and keeps its
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
constexpr int EV_QUEUES = 4 + MAXL;   // flight, next flight, collide, free, cross per level

// Minimum resident CTAs per SM the register allocation must allow (0: let
// the compiler choose).  One CTA of 8 warps keeps the whole particle state in
// registers; the compiler's own choice (two CTAs) spills it to local memory.
#ifndef TRK_EV_MINB
#define TRK_EV_MINB 1
#endif
#if TRK_EV_MINB > 0
#define TRK_EV_BOUNDS __launch_bounds__(EV_BLOCK, TRK_EV_MINB)
#else
#define TRK_EV_BOUNDS __launch_bounds__(EV_BLOCK)
#endif

// slot state fields
enum DField { D_X, D_Y, D_Z, D_U, D_V, D_W, D_IU, D_IV, D_IW, D_TAU, D_PATH, D_HD, D_T0, ND = D_T0 + 3 * MAXL };
enum IField { I_NLEV, I_ONL, I_ONS, I_MAT, I_PIDX, I_EVENT, I_NSEG, I_STATUS, I_HLEV, I_HSURF, I_HSIDE, I_HDIM,
              I_HSIGN, I_HENTRY, I_L0, NI = I_L0 + 6 * MAXL };

struct EvBuf {
    double* dv;
    int* iv;
    unsigned long long* hash;
    unsigned long long* ctr;    // [0] next particle index
    long long T;                // total slots
    __device__ __forceinline__ double& D(int f, int s) const { return dv[(long long)f * T + s]; }
    __device__ __forceinline__ int& I(int f, int s) const { return iv[(long long)f * T + s]; }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t buf_bytes(long long T) {
    return 256 + align256(size_t(T) * ND * 8) + align256(size_t(T) * NI * 4) + align256(size_t(T) * 8);
}

EvBuf make_buf(void* work, long long T) {
    unsigned char* b = static_cast<unsigned char*>(work);
    EvBuf e;
    e.ctr = reinterpret_cast<unsigned long long*>(b);
    size_t off = 256;
    e.dv = reinterpret_cast<double*>(b + off);
    off += align256(size_t(T) * ND * 8);
    e.iv = reinterpret_cast<int*>(b + off);
    off += align256(size_t(T) * NI * 4);
    e.hash = reinterpret_cast<unsigned long long*>(b + off);
    e.T = T;
    return e;
}

__device__ __forceinline__ void load_state(const EvBuf& B, int s, St& st) {
    st.x = B.D(D_X, s); st.y = B.D(D_Y, s); st.z = B.D(D_Z, s);
    st.d.u = B.D(D_U, s); st.d.v = B.D(D_V, s); st.d.w = B.D(D_W, s);
    st.d.iu = B.D(D_IU, s); st.d.iv = B.D(D_IV, s); st.d.iw = B.D(D_IW, s);
    st.tau = B.D(D_TAU, s);
    st.nlev = B.I(I_NLEV, s); st.on_lev = B.I(I_ONL, s); st.on_surf = B.I(I_ONS, s); st.mat = B.I(I_MAT, s);
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        Lv& L = st.lv[l];
        L.tx = B.D(D_T0 + 3 * l, s); L.ty = B.D(D_T0 + 3 * l + 1, s); L.tz = B.D(D_T0 + 3 * l + 2, s);
        L.u = B.I(I_L0 + 6 * l, s); L.cell = B.I(I_L0 + 6 * l + 1, s); L.i = B.I(I_L0 + 6 * l + 2, s);
        L.j = B.I(I_L0 + 6 * l + 3, s); L.k = B.I(I_L0 + 6 * l + 4, s); L.off = B.I(I_L0 + 6 * l + 5, s);
    }
}

__device__ __forceinline__ void store_levels(const EvBuf& B, int s, const St& st) {
    B.I(I_NLEV, s) = st.nlev; B.I(I_ONL, s) = st.on_lev; B.I(I_ONS, s) = st.on_surf; B.I(I_MAT, s) = st.mat;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        const Lv& L = st.lv[l];
        B.D(D_T0 + 3 * l, s) = L.tx; B.D(D_T0 + 3 * l + 1, s) = L.ty; B.D(D_T0 + 3 * l + 2, s) = L.tz;
        B.I(I_L0 + 6 * l, s) = L.u; B.I(I_L0 + 6 * l + 1, s) = L.cell; B.I(I_L0 + 6 * l + 2, s) = L.i;
        B.I(I_L0 + 6 * l + 3, s) = L.j; B.I(I_L0 + 6 * l + 4, s) = L.k; B.I(I_L0 + 6 * l + 5, s) = L.off;
    }
}

__device__ __forceinline__ void store_dir(const EvBuf& B, int s, const St& st) {
    B.D(D_U, s) = st.d.u; B.D(D_V, s) = st.d.v; B.D(D_W, s) = st.d.w;
    B.D(D_IU, s) = st.d.iu; B.D(D_IV, s) = st.d.iv; B.D(D_IW, s) = st.d.iw;
}

__device__ __forceinline__ void load_ctx(const EvBuf& B, int s, Ctx& c, const RunP& rp) {
    const int pidx = B.I(I_PIDX, s);
    c.pid = uint32_t(rp.first_id + uint64_t(uint32_t(pidx)));
    c.event = uint32_t(B.I(I_EVENT, s));
    c.nseg = (long long)(uint32_t)B.I(I_NSEG, s);
    c.path = B.D(D_PATH, s);
    c.hash = B.hash[s];
    c.status = B.I(I_STATUS, s);
}

__device__ __forceinline__ void store_ctx(const EvBuf& B, int s, const Ctx& c) {
    B.I(I_EVENT, s) = int(c.event);
    B.I(I_NSEG, s) = int(uint32_t(c.nseg));
    B.D(D_PATH, s) = c.path;
    B.hash[s] = c.hash;
    B.I(I_STATUS, s) = c.status;
}

// Warp-level append of `v` to `list` when `flag` (all 32 lanes call);
// `count` is warp-uniform and advanced in every lane.
__device__ __forceinline__ void wpush(bool flag, int v, int* list, int& count) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31;
    if (flag) list[count + __popc(m & ((1u << lane) - 1u))] = v;
    count += __popc(m);
}

template <int FLAGS>
__device__ __forceinline__ void finish(const EvBuf& B, int s, const Ctx& c, unsigned long long* rec) {
    if (FLAGS & F_REC) {
        const long long pidx = (long long)(uint32_t)B.I(I_PIDX, s);
        rec[2 * pidx] = c.hash;
        rec[2 * pidx + 1] = (uint64_t(c.nseg) << 32) | uint32_t(c.status);
    }
}

// Each warp owns `slots` particle slots and its own five queues in shared
// memory; warps never synchronise with each other.
template <bool CSG, bool F32, int FLAGS>
__global__ void TRK_EV_BOUNDS k_event(const DevGeom g, const ParticlesView P, long long n, const RunP rp,
                                                    const EvBuf B, int slots, unsigned long long max_rounds,
                                                    unsigned long long* __restrict__ tally,
                                                    unsigned long long* __restrict__ counters,
                                                    unsigned long long* __restrict__ rec) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* base_q = smem + warp * EV_QUEUES * slots;
    int* fly = base_q;
    int* next = base_q + slots;
    int* qc = base_q + 2 * slots;
    int* qf = base_q + 3 * slots;
    int* qx = base_q + 4 * slots;      // MAXL cross queues, one per crossing level
    const int slot0 = (blockIdx.x * (EV_BLOCK / 32) + warp) * slots;
    Counts cnt;
#pragma unroll
    for (int k = 0; k < NCOUNT; ++k) cnt.k[k] = 0;
    for (int k = lane; k < slots; k += 32) qf[k] = slot0 + k;
    int n_fly = 0, n_free = slots;
    bool exhausted = false;
    __syncwarp();
    for (unsigned long long round = 0;; ++round) {
        // ---- refill free slots with new particles --------------------------
        int got = 0;
        unsigned long long first = 0;
        if (!exhausted && n_free > 0) {
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
            int slot = 0;
            if (k < got) {
                slot = qf[n_free - got + k];
                const long long pidx = (long long)first + k;
                Ctx c;
                c.pid = uint32_t(rp.first_id + uint64_t(pidx));
                c.event = 0; c.nseg = 0; c.path = 0.0; c.hash = FNV0; c.status = 0;
                B.I(I_PIDX, slot) = int(pidx);
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
                        B.D(D_X, slot) = s.x; B.D(D_Y, slot) = s.y; B.D(D_Z, slot) = s.z; B.D(D_TAU, slot) = s.tau;
                        store_dir(B, slot, s);
                        store_levels(B, slot, s);
                        ok = true;
                    }
                }
                store_ctx(B, slot, c);
                if (!ok) finish<FLAGS>(B, slot, c, rec);
            }
            wpush(ok, slot, fly, n_fly);
            wpush(k < got && !ok, slot, next, n_park);
        }
        __syncwarp();
        n_free -= got;
        for (int b = 0; b < n_park; b += 32) {
            const int k = b + lane;
            wpush(k < n_park, k < n_park ? next[k] : 0, qf, n_free);
        }
        __syncwarp();
        if (n_fly == 0 && exhausted) break;
        if (round >= max_rounds) {
            if (lane == 0) kernel_status(counters, TRK_E_TIMEOUT);
            break;
        }
        // ---- flight: distance_to_surface, tally, move ----------------------
        int n_cross[MAXL], n_coll = 0;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) n_cross[l] = 0;
        for (int b = 0; b < n_fly; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0;
            if (k < n_fly) {
                slot = fly[k];
                St s;
                load_state(B, slot, s);
                Ctx c;
                load_ctx(B, slot, c, rp);
                Hit h;
                a = step_fly<CSG, F32, FLAGS>(g, s, h, c, rp, tally, cnt, nullptr, nullptr, 0);
                B.D(D_X, slot) = s.x; B.D(D_Y, slot) = s.y; B.D(D_Z, slot) = s.z; B.D(D_TAU, slot) = s.tau;
                store_ctx(B, slot, c);
                if (a == A_CROSS) {
                    B.D(D_HD, slot) = h.d;
                    B.I(I_HLEV, slot) = h.level; B.I(I_HSURF, slot) = h.surf; B.I(I_HSIDE, slot) = h.side;
                    B.I(I_HDIM, slot) = h.dim; B.I(I_HSIGN, slot) = h.dsign; B.I(I_HENTRY, slot) = h.entry;
                }
                if (a == A_DONE) finish<FLAGS>(B, slot, c, rec);
            }
            const bool live = k < n_fly;
            // crossings are queued by level, so each pass runs one code path
            // (array index step, universe search, pin cell test)
            const int hl = (a == A_CROSS) ? B.I(I_HLEV, slot) : -1;
#pragma unroll
            for (int l = 0; l < MAXL; ++l) wpush(live && hl == l, slot, qx + l * slots, n_cross[l]);
            wpush(live && a == A_COLLIDE, slot, qc, n_coll);
            wpush(live && a == A_DONE, slot, qf, n_free);
        }
        __syncwarp();
        // ---- cross_surface, then change_direction ---------------------------
        int n_next = 0;
#pragma unroll 1
        for (int lq = 0; lq < MAXL; ++lq)
        for (int b = 0; b < n_cross[lq]; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0;
            if (k < n_cross[lq]) {
                slot = qx[lq * slots + k];
                St s;
                load_state(B, slot, s);
                Ctx c;
                load_ctx(B, slot, c, rp);
                Hit h;
                h.d = B.D(D_HD, slot);
                h.level = B.I(I_HLEV, slot); h.surf = B.I(I_HSURF, slot); h.side = B.I(I_HSIDE, slot);
                h.dim = B.I(I_HDIM, slot); h.dsign = B.I(I_HSIGN, slot); h.entry = B.I(I_HENTRY, slot);
                a = step_cross<CSG>(g, s, h, c, rp, cnt);
                store_levels(B, slot, s);
                store_dir(B, slot, s);
                store_ctx(B, slot, c);
                if (a == A_DONE) finish<FLAGS>(B, slot, c, rec);
            }
            const bool live = k < n_cross[lq];
            wpush(live && a == A_FLY, slot, next, n_next);
            wpush(live && a == A_DONE, slot, qf, n_free);
        }
        for (int b = 0; b < n_coll; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0;
            if (k < n_coll) {
                slot = qc[k];
                St s;
                s.d.u = B.D(D_U, slot); s.d.v = B.D(D_V, slot); s.d.w = B.D(D_W, slot);
                s.tau = B.D(D_TAU, slot);
                Ctx c;
                load_ctx(B, slot, c, rp);
                a = step_collide(g, s, c, rp, cnt);
                if (a != A_DONE) {
                    store_dir(B, slot, s);
                    B.D(D_TAU, slot) = s.tau;
                    B.I(I_ONL, slot) = -1;
                    B.I(I_ONS, slot) = -1;
                }
                store_ctx(B, slot, c);
                if (a == A_DONE) finish<FLAGS>(B, slot, c, rec);
            }
            const bool live = k < n_coll;
            wpush(live && a == A_FLY, slot, next, n_next);
            wpush(live && a == A_DONE, slot, qf, n_free);
        }
        __syncwarp();
        int* t = fly; fly = next; next = t;
        n_fly = n_next;
    }
    flush_counts(cnt, counters);
}

}  // namespace

namespace trk {

constexpr int EV_WARPS = EV_BLOCK / 32;

int event_grid(int slots) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 1;
    const size_t smem = size_t(EV_QUEUES) * slots * EV_WARPS * sizeof(int);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_event<true, false, 0>, EV_BLOCK, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

size_t event_work_bytes(int slots, int grid) { return buf_bytes((long long)slots * EV_WARPS * grid); }

trk_status launch_event(trk_geom_t g, const ParticlesView& P, long long n, const RunP& rp, bool csg, bool f32,
                        int flags, unsigned long long* tally, unsigned long long* cnt, unsigned long long* rec,
                        void* work, size_t work_bytes, int slots, int grid, int max_rounds_opt, cudaStream_t s) {
    const long long T = (long long)slots * EV_WARPS * grid;
    if (work_bytes < buf_bytes(T) || !work)
        return trk_status(set_error(TRK_E_NOMEM, "run_histories (event): work buffer needs %zu bytes", buf_bytes(T)));
    const EvBuf B = make_buf(work, T);
    cudaError_t e = cudaMemsetAsync(B.ctr, 0, 8, s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_histories (event): %s", cudaGetErrorString(e)));
    const size_t smem = size_t(EV_QUEUES) * slots * EV_WARPS * sizeof(int);
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
