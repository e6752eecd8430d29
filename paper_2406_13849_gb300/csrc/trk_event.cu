// trk_event.cu - persistent event-based kernel (sm_103a).
//
// Paper: Sec. 2.3 (event-based GPU transport: tracking operations run over a
// vector of histories, one operation at a time) on top of Alg. 2-10.
//
// GB300 design.  Each warp owns `slots` particle slots whose state lives in
// the caller's work buffer (one 128-byte record per slot) and keeps its
// own queues of slot indices in shared memory: flight (distance_to_surface +
// move_within_cell + tally), cross (cross_surface + find_cell below, one
// queue per level), collide (change_direction), FP64 redo (FP32-local
// flights too close to call), free.  A round runs refill, then flight, redo,
// cross and collide over full 32-lane batches of their queues (the tail of
// each waits for a later round until the warp's source is exhausted), all
// 32 lanes on one kind of operation, so the warp stays converged where the
// history kernel diverges.  Queue counts are warp-uniform registers advanced by
// ballot/popc; empty slots take new particles from one global counter.  No
// warp ever waits for another (only __syncwarp), and a round limit turns a
// runaway into TRK_E_TIMEOUT.
// Per-particle arithmetic is the history kernel's, so results are the same
// bit for bit.
#include <cstdint>

// the event kernels read the BVH from a shared-memory copy (see k_event)
#ifndef TRK_BVH_SMEM
#define TRK_BVH_SMEM 1
#endif
#include "trk.h"
#include "trk_device.cuh"
#include "trk_internal.h"
#include "trk_event.cuh"
#include "trk_launch.h"

using namespace trk;
using namespace trk::dev;
using namespace trk::ev;

namespace {

// Each warp owns `slots` particle slots and its own queues in shared memory;
// warps never synchronise with each other.
// n_snodes > 0: the geometry's BVH nodes (all n_snodes of them) are copied
// into shared memory after the queues at launch, and every BVH walk of the
// block reads that copy (Sec. 4.3's search, its nodes next to the SM).
template <bool CSG, bool F32, int FLAGS>
__global__ void TRK_EV_BOUNDS k_event(const DevGeom g, const ParticlesView P, long long n, const RunP rp,
                                      const EvBuf B, int slots, unsigned long long max_rounds,
                                      unsigned long long* __restrict__ tally,
                                      unsigned long long* __restrict__ counters,
                                      unsigned long long* __restrict__ rec, int n_snodes, int sort_interval) {
    extern __shared__ QIdx smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#if TRK_BVH_SMEM
    {
        BvhNode* sn = reinterpret_cast<BvhNode*>(smem + EV_QUEUES * slots * (EV_BLOCK / 32));
        const float4* src = reinterpret_cast<const float4*>(g.nodes);
        float4* dst = reinterpret_cast<float4*>(sn);
        for (int k = threadIdx.x; k < 4 * n_snodes; k += EV_BLOCK) dst[k] = __ldg(src + k);
        if (threadIdx.x == 0) s_bvh_nodes = n_snodes > 0 ? sn : nullptr;
        __syncthreads();
    }
#endif
    QIdx* base_q = smem + warp * EV_QUEUES * slots;
    QIdx* qfl = base_q;                  // flight (slot | leaf class << QSLOT_BITS)
    QIdx* qc = base_q + slots;           // collide
    QIdx* qf = base_q + 2 * slots;       // free
    QIdx* qr = base_q + 3 * slots;       // FP32-local flights to redo in FP64
    QIdx* qx = base_q + 4 * slots;       // MAXL cross queues, one per crossing level
    const int slot0 = (blockIdx.x * (EV_BLOCK / 32) + warp) * slots;
#ifndef TRK_EV_SORT
#define TRK_EV_SORT 1
#endif
    const bool sorting = TRK_EV_SORT && sort_interval > 0;
    Counts cnt;
#pragma unroll
    for (int k = 0; k < NCOUNT; ++k) cnt.k[k] = 0;
    for (int k = lane; k < slots; k += 32) qf[k] = QIdx(k);
    // queue counts (warp-uniform); every queue keeps what a pass leaves
    // (batch_run) for the next round
    int n_fly = 0, n_coll = 0, n_redo = 0;
    int n_cross[MAXL];
#pragma unroll
    for (int l = 0; l < MAXL; ++l) n_cross[l] = 0;
    int n_free = slots;
    bool exhausted = false;
    __syncwarp();
    for (unsigned long long round = 0;; ++round) {
        // ---- refill free slots with new particles --------------------------
        // in batches of at least TRK_EV_REFILL_MIN (birth runs the universe
        // searches from the root, whose lanes diverge least when the batches
        // are full), unless the flight queues are running low
        int got = 0;
        unsigned long long first = 0;
        if (!exhausted && n_free > 0 && (n_free >= TRK_EV_REFILL_MIN || n_fly < 32)) {
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
                        unsigned char* r = rec_at<FLAGS>(B, slot);
                        cls = sorting ? flight_class<CSG>(g, s) : 0;
                        D2(r, R_XY) = make_double2(s.x, s.y);
                        D2(r, R_ZT) = make_double2(s.z, s.tau);
                        store_dir(r, s);
                        store_levels<CSG>(g, r, s, 0);
                        store_ctx<FLAGS>(r, int(pidx), c, make_misc(0, s, cls));
                        ok = true;
                    }
                }
                if (!ok) {
                    finish<FLAGS>(pidx, c, rec);
                    trace_tail<FLAGS>(pidx, c, rp);
                    if (FLAGS & F_FISS) fission_out(rp, pidx, 0, 0.0, 0.0, 0.0);
                }
            }
            // failed births park past the collide queue's entries (room:
            // got <= n_free <= slots - n_coll)
            wpush(ok, (slot - slot0) | (cls << QSLOT_BITS), qfl, n_fly);
            wpush(k < got && !ok, slot - slot0, qc + n_coll, n_park);
        }
        __syncwarp();
        n_free -= got;
        for (int b = 0; b < n_park; b += 32) {
            const int k = b + lane;
            wpush(k < n_park, k < n_park ? qc[n_coll + k] : 0, qf, n_free);
        }
        __syncwarp();
        int queued = n_fly + n_coll + n_redo;
        bool full = n_fly >= 32 || n_coll >= 32 || n_redo >= 32;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) {
            queued += n_cross[l];
            full = full || n_cross[l] >= 32;
        }
        if (queued == 0 && exhausted) break;
        // tails run too once the source is exhausted, or when no queue holds
        // a full batch (so every round advances: a full batch, or every
        // queued particle)
        const bool drain = exhausted || !full;
        if (round >= max_rounds) {
            if (lane == 0) kernel_status(counters, TRK_E_TIMEOUT);
            break;
        }
        // ---- flight: distance_to_surface, tally, move ----------------------
        // every sort_interval rounds the flight list is reordered by class
        // (through the free queue's unused tail: slots - n_free >= n_fly)
        if (sorting && n_fly > 32 && round % (unsigned long long)sort_interval == 0) {
            sort_by_class(qfl, n_fly, qf + n_free);
            for (int k = lane; k < n_fly; k += 32) qfl[k] = qf[n_free + k];
            __syncwarp();
        }
        // FP32-local flights that need FP64 (A_REDO) wait in their own queue
        // and are redone in a second pass over full batches, so a warp pays
        // for the FP64 step once per 32 of them rather than once per batch
        // holding one
#pragma unroll 1
        for (int pass = 0; pass < (F32 ? 2 : 1); ++pass) {
        QIdx* list = pass == 0 ? qfl : qr;
        const int n_list = batch_run(pass == 0 ? n_fly : n_redo, drain);
        for (int b = 0; b < n_list; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0, hl = -1;
            if (k < n_list) {
                slot = slot0 + int(unsigned(list[k]) & QSLOT_MASK);
                unsigned char* r = rec_at<FLAGS>(B, slot);
                St s;
                const double2 xy = D2(r, R_XY), zt = D2(r, R_ZT);
                s.x = xy.x; s.y = xy.y; s.z = zt.x; s.tau = zt.y;
                load_dir(r, s);
                Ctx c;
                unsigned misc;
                const int pidx = load_ctx<FLAGS>(r, c, misc, rp);
                int4 su = I4(r, R_SU);
                load_levels<CSG>(g, r, s, misc, su);
                Hit h;
                if (F32 && pass) a = step_flight_fp64_call<CSG, FLAGS>(g, s, h, c, rp, tally, cnt, rp.tr_inst, rp.tr_len, pidx);
                else a = step_fly<CSG, F32, FLAGS, true>(g, s, h, c, rp, tally, cnt, rp.tr_inst, rp.tr_len, pidx);
                if (a == A_REDO) {
                } else if (a == A_DONE) {
                    finish<FLAGS>(pidx, c, rec);
                    trace_tail<FLAGS>(pidx, c, rp);
                    if (FLAGS & F_FISS) fission_out(rp, pidx, 0, 0.0, 0.0, 0.0);
                } else {
                    D2(r, R_XY) = make_double2(s.x, s.y);
                    D2(r, R_ZT) = make_double2(s.z, s.tau);
                    if (a == A_CROSS) {
                        hl = h.level;
                        store_ctx<FLAGS>(r, pidx, c, misc_with_hit(misc, pack_hit(h)));
                        su.y = hit_ref(h);
                        I4(r, R_SU) = su;
                    } else {
                        store_ctx<FLAGS>(r, pidx, c, misc);
                    }
                }
            }
            const bool live = k < n_list;
            // crossings are queued by level, so each pass runs one code path
            // (array index step, universe search, pin cell test)
#pragma unroll
            for (int l = 0; l < MAXL; ++l) wpush(live && hl == l, slot - slot0, qx + l * slots, n_cross[l]);
            wpush(live && a == A_COLLIDE, slot - slot0, qc, n_coll);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
            if (F32) wpush(live && a == A_REDO, slot - slot0, qr, n_redo);
        }
        __syncwarp();
        if (pass == 0) carry_tail(qfl, n_list, n_fly);
        else carry_tail(qr, n_list, n_redo);
        }
        // ---- cross_surface, then change_direction ---------------------------
#pragma unroll 1
        for (int lq = 0; lq < MAXL; ++lq) {
        const int n_list = batch_run(n_cross[lq], drain);
        for (int b = 0; b < n_list; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0, cls = 0;
            if (k < n_list) {
                slot = slot0 + qx[lq * slots + k];
                unsigned char* r = rec_at<FLAGS>(B, slot);
                St s;
                const double2 xy = D2(r, R_XY), zt = D2(r, R_ZT);
                s.x = xy.x; s.y = xy.y; s.z = zt.x; s.tau = zt.y;
                load_dir(r, s);
                Ctx c;
                unsigned misc;
                const int pidx = load_ctx<FLAGS>(r, c, misc, rp);
                const int4 su = I4(r, R_SU);
                load_levels<CSG>(g, r, s, misc, su);
                Hit h;
                unpack_hit(misc_hpack(misc), h);
                hit_from_ref(g, su.y, h);
                h.d = 0.0;
                const unsigned refl0 = cnt.k[TRK_K_REFLECTIONS];
                a = step_cross<CSG>(g, s, h, c, rp, cnt);
                if (a == A_DONE) {
                    finish<FLAGS>(pidx, c, rec);
                    trace_tail<FLAGS>(pidx, c, rp);
                    if (FLAGS & F_FISS) fission_out(rp, pidx, 0, 0.0, 0.0, 0.0);
                } else {
                    cls = sorting ? flight_class<CSG>(g, s) : 0;
                    store_levels<CSG>(g, r, s, 0);
                    store_ctx<FLAGS>(r, pidx, c, make_misc(0, s, cls));
                    if (cnt.k[TRK_K_REFLECTIONS] != refl0) store_dir(r, s);
                }
            }
            const bool live = k < n_list;
            wpush(live && a == A_FLY, (slot - slot0) | (cls << QSLOT_BITS), qfl, n_fly);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
        }
        __syncwarp();
        carry_tail(qx + lq * slots, n_list, n_cross[lq]);
        }
        const int n_crun = batch_run(n_coll, drain);
        for (int b = 0; b < n_crun; b += 32) {
            const int k = b + lane;
            int a = A_DONE, slot = 0, cls = 0;
            if (k < n_crun) {
                slot = slot0 + qc[k];
                unsigned char* r = rec_at<FLAGS>(B, slot);
                St s;
                Ctx c;
                unsigned misc;
                const int pidx = load_ctx<FLAGS>(r, c, misc, rp);
                a = step_collide(g, s, c, rp, cnt);
                if (a == A_DONE) {
                    finish<FLAGS>(pidx, c, rec);
                    trace_tail<FLAGS>(pidx, c, rp);
                    if (FLAGS & F_FISS) {
                        int nf = 0;
                        double fx = 0.0, fy = 0.0, fz = 0.0;
                        if (c.status == TRK_P_ABSORBED) {
                            const double2 xy = D2(r, R_XY), zt = D2(r, R_ZT);
                            fx = xy.x; fy = xy.y; fz = zt.x;
                            nf = fission_sites(g, c.pid, c.event, misc_mat(misc), rp);
                        }
                        fission_out(rp, pidx, nf, fx, fy, fz);
                    }
                } else {
                    store_dir(r, s);
                    const double z = D2(r, R_ZT).x;
                    D2(r, R_ZT) = make_double2(z, s.tau);
                    cls = misc_cls(misc);
                    int4 su = I4(r, R_SU);
                    su.x = -1;
                    I4(r, R_SU) = su;
                    store_ctx<FLAGS>(r, pidx, c, misc_off_surface(misc));
                }
            }
            const bool live = k < n_crun;
            wpush(live && a == A_FLY, (slot - slot0) | (cls << QSLOT_BITS), qfl, n_fly);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
        }
        __syncwarp();
        carry_tail(qc, n_crun, n_coll);
    }
    flush_counts(cnt, counters);
}

}  // namespace

namespace trk {

constexpr int EV_WARPS = EV_BLOCK / 32;

// Resident CTAs per SM: the register budget's minimum (TRK_EV_MINB), capped
// by shared memory.  Deterministic, so the work-buffer size a caller queries
// always matches the launch.
// BVH nodes staged in shared memory per block at most (64 B each); a
// geometry with more nodes walks them from global memory.
constexpr int EV_SMEM_NODES = TRK_BVH_SMEM ? 384 : 0;

int event_grid(int slots) {
    int dev = 0, sms = 152, smem_sm = 228 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    const size_t smem = size_t(EV_QUEUES) * slots * EV_WARPS * sizeof(QIdx) + size_t(EV_SMEM_NODES) * sizeof(BvhNode);
    const int by_smem = int(size_t(smem_sm) / (smem + 1024));
    int per_sm = TRK_EV_MINB > 0 ? TRK_EV_MINB : 1;
    if (per_sm > by_smem) per_sm = by_smem;
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

size_t event_work_bytes(int slots, int grid) { return buf_bytes((long long)slots * EV_WARPS * grid); }

// The slot record packs universes, materials and rect element indices into
// narrow fields; a geometry beyond them is refused before any launch.
trk_status event_fits(trk_geom_t g, bool csg, const char* where) {
    if (g->dg.n_univ > REC_MAX_UNIV || g->n_mat > REC_MAX_MAT || (!csg && g->max_rect_dim > REC_MAX_DIM)) {
        if (!where) return TRK_E_UNSUPPORTED;
        return trk_status(set_error(TRK_E_UNSUPPORTED,
                                    "%s: the event kernels take at most %d universes, %d materials and (array "
                                    "tracker) %d elements per array axis",
                                    where, REC_MAX_UNIV, REC_MAX_MAT, REC_MAX_DIM));
    }
    return TRK_OK;
}

trk_status launch_event(trk_geom_t g, const ParticlesView& P, long long n, const RunP& rp, bool csg, bool f32,
                        int flags, unsigned long long* tally, unsigned long long* cnt, unsigned long long* rec,
                        void* work, size_t work_bytes, int slots, int grid, int max_rounds_opt, int sort_interval,
                        cudaStream_t s) {
    const long long T = (long long)slots * EV_WARPS * grid;
    const trk_status fit = event_fits(g, csg, "run_histories (event)");
    if (fit != TRK_OK) return fit;
    if (work_bytes < buf_bytes(T) || !work)
        return trk_status(set_error(TRK_E_NOMEM, "run_histories (event): work buffer needs %zu bytes", buf_bytes(T)));
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return trk_status(set_error(TRK_E_INVALID, "run_histories (event): work buffer must be 256-byte aligned"));
    const EvBuf B = make_buf(work, T);
    cudaError_t e = cudaMemsetAsync(B.ctr, 0, 8, s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_histories (event): %s", cudaGetErrorString(e)));
    const int n_snodes = (g->dg.accel == 0 && g->n_nodes <= EV_SMEM_NODES) ? g->n_nodes : 0;
    const size_t smem = size_t(EV_QUEUES) * slots * EV_WARPS * sizeof(QIdx) + size_t(n_snodes) * sizeof(BvhNode);
    // a particle takes at most 3 (max_segments + 2) queue steps (flight,
    // redo, cross or collide); until its source runs out a warp runs at
    // least one full batch of 32 steps a round, after that every queued
    // particle advances every round
    const unsigned long long per_warp = (unsigned long long)(n / (T / slots) + slots + 1);
    unsigned long long max_rounds = (rp.max_segments + 2ULL) * (per_warp / 32ULL + 2ULL) * 4ULL;
    if (max_rounds_opt > 0) max_rounds = (unsigned long long)max_rounds_opt;
#define TRK_EV(C, F32V, F)                                                                                   \
    do {                                                                                                     \
        auto k = k_event<C, F32V, F>;                                                                        \
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); \
        k<<<grid, EV_BLOCK, smem, s>>>(g->dg, P, n, rp, B, slots, max_rounds, tally, cnt, rec, n_snodes,     \
                                        sort_interval);                                                     \
    } while (0)
    if (f32) {
#ifndef TRK_EXACT
        if (csg) {
            if (flags & F_TRACE) TRK_EV(true, true, F_TRACE);
            else if (flags & F_REC) TRK_EV(true, true, F_REC);
            else TRK_EV(true, true, 0);
        } else {
            if (flags & F_TRACE) TRK_EV(false, true, F_TRACE);
            else if (flags & F_REC) TRK_EV(false, true, F_REC);
            else TRK_EV(false, true, 0);
        }
#endif
    } else if (csg) {
        switch (flags) {
            case F_TRACE: TRK_EV(true, false, F_TRACE); break;
            case 0: TRK_EV(true, false, 0); break;
            case F_REC: TRK_EV(true, false, F_REC); break;
            case F_CUT: TRK_EV(true, false, F_CUT); break;
            case F_MESH: TRK_EV(true, false, F_MESH); break;
            case F_MESH | F_REC: TRK_EV(true, false, F_MESH | F_REC); break;
            case F_FISS: TRK_EV(true, false, F_FISS); break;
            case F_FISS | F_MESH: TRK_EV(true, false, F_FISS | F_MESH); break;
            default: TRK_EV(true, false, F_REC | F_CUT); break;
        }
    } else {
        switch (flags) {
            case F_TRACE: TRK_EV(false, false, F_TRACE); break;
            case 0: TRK_EV(false, false, 0); break;
            case F_REC: TRK_EV(false, false, F_REC); break;
            case F_CUT: TRK_EV(false, false, F_CUT); break;
            case F_MESH: TRK_EV(false, false, F_MESH); break;
            case F_MESH | F_REC: TRK_EV(false, false, F_MESH | F_REC); break;
            case F_FISS: TRK_EV(false, false, F_FISS); break;
            case F_FISS | F_MESH: TRK_EV(false, false, F_FISS | F_MESH); break;
            default: TRK_EV(false, false, F_REC | F_CUT); break;
        }
    }
#undef TRK_EV
    e = cudaGetLastError();
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_histories (event): %s", cudaGetErrorString(e)));
    return TRK_OK;
}

}  // namespace trk
