// batch.cu - many independent geometries and particle populations in one
// persistent launch (sm_103a), plus the autotuner that picks its launch shape.
//
// Paper: the tracking loop of Alg. 2 run over many problems at once; the
// paper runs one problem per GPU, this is the serving-style form of it.
//
// Design.  The caller's work buffer holds a device table: one entry per
// geometry (its flattened geometry view, particle buffer, tally, counters,
// tracker) and the prefix sums of its particle chunks.  History mode: warps
// pull chunk indices from one global counter; a chunk is `chunk` particles
// of a single geometry, so the geometry and the tracker type are uniform
// across the warp (warp-level dispatch: one branch per chunk, never per
// particle), and chunks are numbered with every rect-tracker geometry before
// every CSG one, so neighbouring chunks share code.  Event mode: per-geometry
// chunk counters (see k_batched_ev).  run_batched issues only memsets, the
// kernels and, for an array-tracker batch in event mode, a fork/join with a
// side stream: after batch_upload it can be captured in a CUDA graph and
// replayed.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "trk.h"
#include "trk_device.cuh"
#include "trk_internal.h"
#include "trk_event.cuh"
#include "trk_launch.h"

using namespace trk;
using namespace trk::dev;

namespace {

struct BatchEntry {
    DevGeom g;
    ParticlesView P;
    unsigned long long* tally;
    unsigned long long* counters;
    unsigned long long* records;
    long long n;
    long long first_chunk;   // prefix sum of chunks before this entry (in chunk order)
    long long part_first;    // event mode: particles before this entry among the same tracker's entries
    int csg;
    int pad;
};

// Population order of all entries, for a single event launch over them:
// entry index and the particles of the entries before it in that order.
struct EvOrder {
    long long part_first;
    int entry, pad;
};

struct BatchHeader {
    unsigned long long next_chunk;
    unsigned long long total_chunks;
    int n_geom;
    int chunk;
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

template <bool CSG, bool F32, int FLAGS>
__device__ __forceinline__ void run_chunk(const BatchEntry& E, long long a, long long b, const RunP& rp, Counts& cnt) {
    for (long long i = a + (threadIdx.x & 31); i < b; i += 32) {
        Ctx c;
        c.pid = uint32_t(rp.first_id + uint64_t(i));
        c.event = 0; c.nseg = 0; c.path = 0.0; c.hash = FNV0; c.status = 0;
        const int pst = E.P.status[i];
        if (pst != 0) {
            c.status = pst;
            cnt.k[TRK_K_SOURCE]++;
        } else {
            St s;
            load_birth(E.g, E.P, i, s);
            if (find_from<CSG>(E.g, s, 0) != 0) {
                c.status = TRK_E_LOST;
                cnt.k[TRK_K_LOST]++;
            } else {
                for (;;) {
                    Hit h;
                    int act = step_fly<CSG, F32, FLAGS>(E.g, s, h, c, rp, E.tally, cnt, nullptr, nullptr, 0);
                    if (act == A_DONE) break;
                    act = (act == A_CROSS) ? step_cross<CSG>(E.g, s, h, c, rp, cnt) : step_collide(E.g, s, c, rp, cnt);
                    if (act == A_DONE) break;
                }
            }
        }
        if ((FLAGS & F_REC) && E.records) {
            E.records[2 * i] = c.hash;
            E.records[2 * i + 1] = (uint64_t(c.nseg) << 32) | uint32_t(c.status);
        }
    }
}

template <bool F32, int FLAGS>
__global__ void __launch_bounds__(128) k_batched(BatchHeader* __restrict__ hdr, const BatchEntry* __restrict__ table,
                                                const RunP rp) {
    const int lane = threadIdx.x & 31;
    const int ng = hdr->n_geom;
    const int chunk = hdr->chunk;
    const unsigned long long total = hdr->total_chunks;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&hdr->next_chunk, 1ULL);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= total) break;
        // entry holding chunk c: last entry with first_chunk <= c
        int lo = 0, hi = ng - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)table[mid].first_chunk <= c) lo = mid;
            else hi = mid - 1;
        }
        const BatchEntry& E = table[lo];
        const long long a = (long long)(c - (unsigned long long)E.first_chunk) * chunk;
        const long long b = a + chunk < E.n ? a + chunk : E.n;
        Counts cnt;
#pragma unroll
        for (int k = 0; k < NCOUNT; ++k) cnt.k[k] = 0;
        if (E.csg) run_chunk<true, F32, FLAGS>(E, a, b, rp, cnt);
        else run_chunk<false, F32, FLAGS>(E, a, b, rp, cnt);
        __syncwarp();
        flush_counts(cnt, E.counters);
    }
}

// ---------------------------------------------------------------------------
// Event mode: each warp runs the event loop of the single-geometry event
// kernel (slot records, queues by operation) over chunks of one geometry at
// a time.  Chunks come from per-entry counters: a warp starts on the entry
// its share of the launch's particle range falls in (warps spread over the
// entries in proportion to their particles) and keeps pulling that entry's
// chunks, refilling without a break; when the entry runs out it takes the
// entry with the most chunks left, whose first chunk waits until the warp's
// slots have drained, so the geometry and tracker stay warp-uniform.  An
// AUTO or CSG batch is one launch (the CSG tracker for every entry); a batch
// created for the array tracker runs its array and CSG entries as two.
// ---------------------------------------------------------------------------
using namespace trk::ev;
#ifndef TRK_BATCH_SM_GROUP
#define TRK_BATCH_SM_GROUP 1
#endif
constexpr int BEV_QUEUES = 4 + MAXL;   // flight, collide, free, FP64 redo, cross per level

template <bool CSG, bool F32, int FLAGS>
__global__ void TRK_EV_BOUNDS k_batched_ev(BatchHeader* __restrict__ hdr, const BatchEntry* __restrict__ table,
                                           unsigned long long* __restrict__ ectr,
                                           const RunP rp, const EvBuf B, int slots, int e_begin, int e_end,
                                           long long side_parts, const EvOrder* __restrict__ evo,
                                           unsigned long long max_rounds, int sort_interval, int per_sm) {
    extern __shared__ QIdx smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    QIdx* base_q = smem + warp * BEV_QUEUES * slots;
    QIdx* fly = base_q;                  // slot | leaf class << QSLOT_BITS
    QIdx* qc = base_q + slots;           // collide
    QIdx* qf = base_q + 2 * slots;       // free
    QIdx* qr = base_q + 3 * slots;       // FP32-local flights to redo in FP64
    QIdx* qx = base_q + 4 * slots;       // cross, one queue per level
    const bool sorting = sort_interval > 0;
    const int slot0 = (blockIdx.x * (EV_BLOCK / 32) + warp) * slots;
    const long long chunk = hdr->chunk;
    // the entry this warp starts on: warps are spread over the entries in
    // proportion to their particles (the warp's share of the side's particle
    // range), so most warps work through chunks of one geometry and switch
    // (draining their slots) only when it runs out
    // (evo: a launch over all entries takes them in population order instead
    // of the table's)
    int pref = e_begin;
    {
        const long long W = (long long)gridDim.x * (EV_BLOCK / 32);
#if TRK_BATCH_SM_GROUP
        // the CTAs of one SM (blocks b, b + nsm, ... of the first wave) take
        // neighbouring shares, so an SM's warps mostly track one geometry
        const int nsm = gridDim.x / per_sm;
        const long long gw = ((long long)(blockIdx.x % nsm) * per_sm + blockIdx.x / nsm) * (EV_BLOCK / 32) + warp;
#else
        const long long gw = (long long)blockIdx.x * (EV_BLOCK / 32) + warp;
#endif
        const long long target = (long long)(((double)gw + 0.5) * (double)side_parts / (double)W);
        int lo = e_begin, hi = e_end - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((evo ? evo[mid].part_first : table[mid].part_first) <= target) lo = mid;
            else hi = mid - 1;
        }
        pref = evo ? evo[lo].entry : lo;
    }
    Counts cnt;
#pragma unroll
    for (int k = 0; k < NCOUNT; ++k) cnt.k[k] = 0;
    for (int k = lane; k < slots; k += 32) qf[k] = QIdx(k);
    // queue counts (warp-uniform); every queue keeps what a pass leaves
    // (batch_run) for the next round
    int n_fly = 0, n_coll = 0, n_redo = 0, n_free = slots;
    int n_cross[MAXL];
#pragma unroll
    for (int l = 0; l < MAXL; ++l) n_cross[l] = 0;
    int ge = -1;                   // current entry, warp-uniform
    long long pn = 0, pb = 0;      // next particle and end of the current chunk
    int pend_e = -1;               // entry and chunk pulled, waiting to start
    long long pend_c = 0;
    bool exhausted = false;
    __syncwarp();
    for (unsigned long long round = 0;; ++round) {
        // ---- chunks: pull the next one when the current is used up ----------
        if (pn >= pb && pend_e < 0 && !exhausted) {
            // the next chunk of the preferred entry; when it has none left,
            // of the entry with the most chunks left (the counters read
            // lane by lane), so the warps that finish early help the
            // geometries that take longest
            int e = pref;
            long long c = -1;
            for (int attempt = 0; attempt < 2 * (e_end - e_begin) + 1 && e >= 0; ++attempt) {
                unsigned long long v = 0;
                if (lane == 0) v = atomicAdd(ectr + e, 1ULL);
                v = __shfl_sync(0xffffffffu, v, 0);
                if ((long long)v < (table[e].n + chunk - 1) / chunk) { c = (long long)v; break; }
                long long best_left = 0;
                int best = -1;
                for (int t = e_begin + lane; t < e_end; t += 32) {
                    const long long nch = (table[t].n + chunk - 1) / chunk;
                    const long long taken = (long long)*reinterpret_cast<volatile unsigned long long*>(ectr + t);
                    const long long left = nch - (taken < nch ? taken : nch);
                    if (left > best_left) { best_left = left; best = t; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long l2 = __shfl_down_sync(0xffffffffu, best_left, o);
                    const int b2 = __shfl_down_sync(0xffffffffu, best, o);
                    if (l2 > best_left || (l2 == best_left && b2 >= 0 && (best < 0 || b2 < best))) {
                        best_left = l2;
                        best = b2;
                    }
                }
                e = __shfl_sync(0xffffffffu, best, 0);
            }
            if (c < 0) exhausted = true;
            else { pend_e = e; pend_c = c; pref = e; }
        }
        int queued = n_fly + n_coll + n_redo;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) queued += n_cross[l];
        if (pend_e >= 0) {
            const int e = pend_e;
            if (e == ge || queued == 0) {
                if (e != ge) {
                    if (ge >= 0) flush_counts(cnt, table[ge].counters);
#pragma unroll
                    for (int k = 0; k < NCOUNT; ++k) cnt.k[k] = 0;
                    ge = e;
                }
                pn = pend_c * chunk;
                pb = pn + chunk < table[e].n ? pn + chunk : table[e].n;
                pend_e = -1;
            }
        }
        if (ge < 0) break;   // no chunk at all for this warp
        const BatchEntry& E = table[ge];
        const DevGeom& g = E.g;
        unsigned long long* rec = (FLAGS & F_REC) ? E.records : nullptr;
        // ---- refill free slots from the current chunk ------------------------
        int got = 0;
        const long long first = pn;
        if (n_free > 0 && pn < pb && (n_free >= TRK_BEV_REFILL_MIN || n_fly < 32)) {
            got = pb - pn < (long long)n_free ? int(pb - pn) : n_free;
            pn += got;
        }
        int n_park = 0;
        for (int b = 0; b < got; b += 32) {
            const int k = b + lane;
            bool ok = false;
            int slot = 0, cls = 0;
            if (k < got) {
                slot = slot0 + qf[n_free - got + k];
                const long long pidx = first + k;
                Ctx c;
                c.pid = uint32_t(rp.first_id + uint64_t(pidx));
                c.event = 0; c.nseg = 0; c.path = 0.0; c.hash = FNV0; c.status = 0;
                const int pst = E.P.status[pidx];
                if (pst != 0) {
                    c.status = pst;
                    cnt.k[TRK_K_SOURCE]++;
                } else {
                    St s;
                    load_birth(g, E.P, pidx, s);
                    if (find_from<CSG>(g, s, 0) != 0) {
                        c.status = TRK_E_LOST;
                        cnt.k[TRK_K_LOST]++;
                    } else {
                        unsigned char* r = rec_at<FLAGS>(B, slot);
                        D2(r, R_XY) = make_double2(s.x, s.y);
                        D2(r, R_ZT) = make_double2(s.z, s.tau);
                        store_dir(r, s);
                        store_levels<CSG>(g, r, s, 0);
                        cls = sorting ? flight_class<CSG>(g, s) : 0;
                        store_ctx<FLAGS>(r, int(pidx), c, make_misc(0, s, cls));
                        ok = true;
                    }
                }
                if (!ok && rec) finish<FLAGS>(pidx, c, rec);
            }
            // failed births park past the collide queue's entries (room:
            // got <= n_free <= slots - n_coll)
            wpush(ok, (slot - slot0) | (cls << QSLOT_BITS), fly, n_fly);
            wpush(k < got && !ok, slot - slot0, qc + n_coll, n_park);
        }
        __syncwarp();
        n_free -= got;
        queued += got - n_park;
        for (int b = 0; b < n_park; b += 32) {
            const int k = b + lane;
            wpush(k < n_park, k < n_park ? qc[n_coll + k] : 0, qf, n_free);
        }
        __syncwarp();
        if (queued == 0 && exhausted && pend_e < 0 && pn >= pb) break;
        bool full = n_fly >= 32 || n_coll >= 32 || n_redo >= 32;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) full = full || n_cross[l] >= 32;
        // tails run too when the chunk is used up and no more of this
        // geometry follows (the source is exhausted, or the next chunk waits
        // for the slots to drain), or when no queue holds a full batch (so
        // every round advances: a full batch, or every queued particle)
        const bool drain = (pn >= pb && (exhausted || pend_e >= 0)) || !full;
        if (round >= max_rounds) {
            if (lane == 0) kernel_status(E.counters, TRK_E_TIMEOUT);
            break;
        }
        // ---- flight ------------------------------------------------------------
        // every sort_interval rounds the flight list is reordered by class
        // (through the free queue's unused tail: slots - n_free >= n_fly)
        if (sorting && n_fly > 32 && round % (unsigned long long)sort_interval == 0) {
            sort_by_class(fly, n_fly, qf + n_free);
            for (int k = lane; k < n_fly; k += 32) fly[k] = qf[n_free + k];
            __syncwarp();
        }
        // FP32-local flights that need FP64 (A_REDO) wait in their own queue
        // and are redone in a second pass over full batches (one FP64 step
        // per 32 of them, not per batch holding one)
#pragma unroll 1
        for (int pass = 0; pass < (F32 ? 2 : 1); ++pass) {
        QIdx* list = pass == 0 ? fly : qr;
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
                if (F32 && pass) a = step_flight_fp64_call<CSG, FLAGS>(g, s, h, c, rp, E.tally, cnt, nullptr, nullptr, 0);
                else a = step_fly<CSG, F32, FLAGS, true>(g, s, h, c, rp, E.tally, cnt, nullptr, nullptr, 0);
                if (a == A_REDO) {
                } else if (a == A_DONE) {
                    if (rec) finish<FLAGS>(pidx, c, rec);
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
#pragma unroll
            for (int l = 0; l < MAXL; ++l) wpush(live && hl == l, slot - slot0, qx + l * slots, n_cross[l]);
            wpush(live && a == A_COLLIDE, slot - slot0, qc, n_coll);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
            if (F32) wpush(live && a == A_REDO, slot - slot0, qr, n_redo);
        }
        __syncwarp();
        if (pass == 0) carry_tail(fly, n_list, n_fly);
        else carry_tail(qr, n_list, n_redo);
        }
        // ---- cross_surface, then change_direction -------------------------------
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
                    if (rec) finish<FLAGS>(pidx, c, rec);
                } else {
                    cls = sorting ? flight_class<CSG>(g, s) : 0;
                    store_levels<CSG>(g, r, s, 0);
                    store_ctx<FLAGS>(r, pidx, c, make_misc(0, s, cls));
                    if (cnt.k[TRK_K_REFLECTIONS] != refl0) store_dir(r, s);
                }
            }
            const bool live = k < n_list;
            wpush(live && a == A_FLY, (slot - slot0) | (cls << QSLOT_BITS), fly, n_fly);
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
                    if (rec) finish<FLAGS>(pidx, c, rec);
                } else {
                    store_dir(r, s);
                    const double z = D2(r, R_ZT).x;
                    D2(r, R_ZT) = make_double2(z, s.tau);
                    int4 su = I4(r, R_SU);
                    su.x = -1;
                    I4(r, R_SU) = su;
                    cls = misc_cls(misc);
                    store_ctx<FLAGS>(r, pidx, c, misc_off_surface(misc));
                }
            }
            const bool live = k < n_crun;
            wpush(live && a == A_FLY, (slot - slot0) | (cls << QSLOT_BITS), fly, n_fly);
            wpush(live && a == A_DONE, slot - slot0, qf, n_free);
        }
        __syncwarp();
        carry_tail(qc, n_crun, n_coll);
    }
    if (ge >= 0) flush_counts(cnt, table[ge].counters);
}

}  // namespace

// Host object behind trk_batch_t.
struct trk_batch {
    std::vector<BatchEntry> entries;   // in chunk order (rect trackers first)
    std::vector<int> order;            // entries[k] is input geometry order[k]
    int n_geom = 0;
    int chunk = 0;                     // chunk size the uploaded table was built for
    bool uploaded = false;
    int event_unfit = -1;              // first geometry the event kernels' slot record cannot hold
    int event_unfit_csg = -1;          // the same for the CSG tracker on every entry
    bool auto_tracker = false;         // created with TRK_TRACKER_AUTO
    void* work = nullptr;
    size_t work_bytes = 0;
    unsigned magic = 0;
    // event mode: the CSG-tracker launch runs on a second stream, forked
    // from and joined to the caller's, so that it fills the SMs the
    // array-tracker launch's last warps leave idle (created at first use)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~trk_batch() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
    }
};
constexpr unsigned TRK_BATCH_MAGIC = 0x74726b62u;

namespace {

bool valid_batch(trk_batch_t b) { return b && b->magic == TRK_BATCH_MAGIC; }

int sm_count_b() {
    int dev = 0, v = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
}

size_t evo_offset(int n) { return a256(sizeof(BatchHeader)) + a256(size_t(n) * sizeof(BatchEntry)); }
// header, entries, the entries' population order
size_t table_bytes(int n) { return evo_offset(n) + a256(size_t(n) * sizeof(EvOrder)); }

// Event mode: per-entry chunk counters after the table, then slot records,
// `slots` per warp, one set for each of the two launches (they may run at
// the same time).
size_t counters_bytes(int n) { return a256(size_t(n) * sizeof(unsigned long long)); }
size_t event_bytes(int n, int slots) {
    return table_bytes(n) + counters_bytes(n) + 2 * event_work_bytes(slots, event_grid(slots));
}
constexpr int BEV_MAX_SLOTS = 512;

}  // namespace

namespace {

// Event mode: the rect-tracker entries [0, split) and the CSG ones
// [split, total) as two launches of the batched event kernel, the second on
// the batch's side stream between a fork and a join event (graph capture
// records the same fork and join), each with its own slot records.
trk_status run_batched_event(trk_batch_t b, void* dev_work, const trk_run_opts& o, const RunP& rp, bool f32, bool rec,
                             cudaStream_t s) {
    const int slots = o.queue_depth > 0 ? o.queue_depth : 256;
    if (slots < 32 || slots > BEV_MAX_SLOTS) return trk_status(set_error(TRK_E_INVALID, "run_batched: queue_depth must be in [32, 512]"));
    if (o.max_rounds < 0) return trk_status(set_error(TRK_E_INVALID, "run_batched: max_rounds must be >= 0"));
    if (o.sort_interval < 0) return trk_status(set_error(TRK_E_INVALID, "run_batched: sort_interval must be >= 0"));
    // AUTO: the CSG tracker for every entry, one launch (its kernel measured
    // 5% faster on the 64-geometry batch than the array-tracker launch with
    // the CSG one beside it: one kernel's code in the instruction caches);
    // the history kernels keep the per-entry choice
    const bool all_csg = b->auto_tracker;
    const int unfit = all_csg ? b->event_unfit_csg : b->event_unfit;
    if (unfit >= 0)
        return trk_status(set_error(TRK_E_UNSUPPORTED, "run_batched (event): geometry %d does not fit the event kernels' "
                                    "slot record (at most %d universes, %d materials, %d elements per array axis)",
                                    unfit, ev::REC_MAX_UNIV, ev::REC_MAX_MAT, ev::REC_MAX_DIM));
    const int grid = event_grid(slots);
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = grid % sms == 0 && grid >= sms ? grid / sms : 1;
    const size_t need = event_bytes(b->n_geom, slots);
    if (b->work_bytes < need)
        return trk_status(set_error(TRK_E_NOMEM, "run_batched (event): work buffer needs %zu bytes", need));
    BatchHeader* hdr = static_cast<BatchHeader*>(dev_work);
    const BatchEntry* table = reinterpret_cast<const BatchEntry*>(static_cast<unsigned char*>(dev_work) + a256(sizeof(BatchHeader)));
    const long long T = (long long)slots * (EV_BLOCK / 32) * grid;
    unsigned long long* ectr =
        reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(dev_work) + table_bytes(b->n_geom));
    unsigned char* rec_base = static_cast<unsigned char*>(dev_work) + table_bytes(b->n_geom) + counters_bytes(b->n_geom);
    const EvOrder* evo = reinterpret_cast<const EvOrder*>(static_cast<unsigned char*>(dev_work) + evo_offset(b->n_geom));
    const EvBuf B0 = make_buf(rec_base, T);
    const EvBuf B1 = make_buf(rec_base + event_work_bytes(slots, grid), T);
    cudaError_t e = cudaMemsetAsync(ectr, 0, size_t(b->n_geom) * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_batched: %s", cudaGetErrorString(e)));
    if (!b->side) {
        if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess)
            return trk_status(set_error(TRK_E_CUDA, "run_batched: cannot create the side stream"));
    }
    // entries [0, n_rect) run with the array tracker, [n_rect, n_geom) with CSG
    int n_rect = 0;
    long long npart = 0, parts_side[2] = {0, 0};
    for (auto& en : b->entries) {
        if (!en.csg) ++n_rect;
        npart += en.n;
        parts_side[en.csg ? 1 : 0] += en.n;
    }
    if (all_csg) {
        n_rect = 0;
        parts_side[0] = 0;
        parts_side[1] = npart;
    }
    // a particle takes at most 3 (max_segments + 2) queue steps; outside a
    // drain a warp runs at least one full batch of 32 of them a round
    unsigned long long max_rounds = (rp.max_segments + 2ULL) * (unsigned long long)(npart / 32 + 2) * 4ULL;
    if (o.max_rounds > 0) max_rounds = (unsigned long long)o.max_rounds;
    const size_t smem = size_t(BEV_QUEUES) * slots * (EV_BLOCK / 32) * sizeof(QIdx);
    // side 1 waits for everything before it on s (the counters' reset)
    const bool both = n_rect > 0 && n_rect < b->n_geom;
    if (both) {
        if (cudaEventRecord(b->fork, s) != cudaSuccess || cudaStreamWaitEvent(b->side, b->fork, 0) != cudaSuccess)
            return trk_status(set_error(TRK_E_CUDA, "run_batched: fork failed"));
    }
    auto launch = [&](auto kernel, int side, int e0, int e1) {
        if (e1 <= e0) return;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        cudaStream_t st = (side == 1 && both) ? b->side : s;
        kernel<<<grid, EV_BLOCK, smem, st>>>(hdr, table, ectr, rp, side == 1 ? B1 : B0, slots, e0, e1,
                                             parts_side[side], all_csg ? evo : nullptr, max_rounds,
                                             o.sort_interval, per_sm);
    };
    const int split = n_rect, total = b->n_geom;
    if (f32) {
#ifndef TRK_EXACT
        if (rec) { launch(k_batched_ev<false, true, F_REC>, 0, 0, split); launch(k_batched_ev<true, true, F_REC>, 1, split, total); }
        else { launch(k_batched_ev<false, true, 0>, 0, 0, split); launch(k_batched_ev<true, true, 0>, 1, split, total); }
#endif
    } else {
        if (rec) { launch(k_batched_ev<false, false, F_REC>, 0, 0, split); launch(k_batched_ev<true, false, F_REC>, 1, split, total); }
        else { launch(k_batched_ev<false, false, 0>, 0, 0, split); launch(k_batched_ev<true, false, 0>, 1, split, total); }
    }
    if (both) {
        if (cudaEventRecord(b->join, b->side) != cudaSuccess || cudaStreamWaitEvent(s, b->join, 0) != cudaSuccess)
            return trk_status(set_error(TRK_E_CUDA, "run_batched: join failed"));
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_batched: %s", cudaGetErrorString(e)));
    return TRK_OK;
}

}  // namespace

extern "C" {

trk_status batch_create(const trk_geom_t* geoms, int n_geom, const void* const* dev_particles,
                        const int64_t* counts, uint64_t* const* dev_tallies, uint64_t* dev_counters,
                        uint64_t* const* dev_records, int tracker, trk_batch_t* out) {
    if (!geoms || n_geom <= 0 || !dev_particles || !counts || !dev_tallies || !dev_counters || !out)
        return trk_status(set_error(TRK_E_INVALID, "batch_create: null argument or n_geom <= 0"));
    if (tracker != TRK_TRACKER_RECT && tracker != TRK_TRACKER_CSG && tracker != TRK_TRACKER_AUTO)
        return trk_status(set_error(TRK_E_INVALID, "batch_create: unknown tracker %d", tracker));
    trk_batch* b = new trk_batch;
    std::vector<int> idx(static_cast<size_t>(n_geom), 0);
    for (int k = 0; k < n_geom; ++k) {
        trk_geom_t g = geoms[k];
        if (!g || g->magic != TRK_GEOM_MAGIC || counts[k] < 0 || counts[k] > (int64_t(1) << 31) ||
            (counts[k] > 0 && (!dev_particles[k] || !dev_tallies[k]))) {
            delete b;
            return trk_status(set_error(TRK_E_INVALID, "batch_create: entry %d invalid", k));
        }
        if (tracker == TRK_TRACKER_RECT && !g->rect_ok) {
            delete b;
            return trk_status(set_error(TRK_E_UNSUPPORTED, "batch_create: entry %d: array tracker not available", k));
        }
        idx[size_t(k)] = k;
    }
    auto use_csg = [&](int k) {
        if (tracker == TRK_TRACKER_CSG) return true;
        return !geoms[k]->rect_ok || geoms[k]->has_hex != 0;
    };
    // array-tracker geometries first (the event mode's two launches take
    // contiguous ranges of entries, and history-mode warps keep to one
    // tracker's code), larger populations first within a type; the event
    // mode's single CSG launch of an AUTO batch reads its own population
    // order (evo, batch_upload)
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) {
        if (use_csg(a) != use_csg(c)) return !use_csg(a);
        return counts[a] > counts[c];
    });
    for (int k : idx) {
        BatchEntry e;
        std::memset(&e, 0, sizeof e);
        e.g = geoms[k]->dg;
        const long long n = counts[k];
        const double* base = static_cast<const double*>(dev_particles[k]);
        e.P.x = base; e.P.y = base + n; e.P.z = base + 2 * n; e.P.u = base + 3 * n; e.P.v = base + 4 * n;
        e.P.w = base + 5 * n; e.P.tau = base + 6 * n; e.P.status = reinterpret_cast<const int*>(base + 7 * n);
        e.tally = reinterpret_cast<unsigned long long*>(dev_tallies[k]);
        e.counters = reinterpret_cast<unsigned long long*>(dev_counters + size_t(k) * TRK_NCOUNTERS);
        e.records = dev_records ? reinterpret_cast<unsigned long long*>(dev_records[k]) : nullptr;
        e.n = n;
        e.csg = use_csg(k) ? 1 : 0;
        if (b->event_unfit < 0 && event_fits(geoms[k], e.csg != 0, nullptr) != TRK_OK) b->event_unfit = k;
        if (b->event_unfit_csg < 0 && event_fits(geoms[k], true, nullptr) != TRK_OK) b->event_unfit_csg = k;
        b->entries.push_back(e);
        b->order.push_back(k);
    }
    b->n_geom = n_geom;
    b->auto_tracker = tracker == TRK_TRACKER_AUTO;
    b->magic = TRK_BATCH_MAGIC;
    *out = b;
    return TRK_OK;
}

trk_status batch_destroy(trk_batch_t b) {
    if (!valid_batch(b)) return trk_status(set_error(TRK_E_INVALID, "batch_destroy: invalid handle"));
    b->magic = 0;
    delete b;
    return TRK_OK;
}

trk_status batch_work_bytes(trk_batch_t b, size_t* bytes) {
    if (!valid_batch(b) || !bytes) return trk_status(set_error(TRK_E_INVALID, "batch_work_bytes: bad arguments"));
    *bytes = event_bytes(b->n_geom, BEV_MAX_SLOTS);
    return TRK_OK;
}

trk_status batch_upload(trk_batch_t b, void* dev_work, size_t work_bytes, int chunk, void* stream) {
    if (!valid_batch(b) || !dev_work) return trk_status(set_error(TRK_E_INVALID, "batch_upload: bad arguments"));
    if (work_bytes < table_bytes(b->n_geom)) return trk_status(set_error(TRK_E_NOMEM, "batch_upload: work buffer too small"));
    if ((reinterpret_cast<uintptr_t>(dev_work) & 255) != 0)
        return trk_status(set_error(TRK_E_INVALID, "batch_upload: work buffer must be 256-byte aligned"));
    if (chunk <= 0) chunk = 512;
    if (chunk < 32 || chunk > (1 << 20)) return trk_status(set_error(TRK_E_INVALID, "batch_upload: chunk must be in [32, 2^20]"));
    long long total = 0, pf[2] = {0, 0};
    for (auto& e : b->entries) {
        e.first_chunk = total;
        total += (e.n + chunk - 1) / chunk;
        e.part_first = pf[e.csg ? 1 : 0];
        pf[e.csg ? 1 : 0] += e.n;
    }
    std::vector<unsigned char> img(table_bytes(b->n_geom), 0);
    BatchHeader h;
    std::memset(&h, 0, sizeof h);
    h.next_chunk = 0;
    h.total_chunks = (unsigned long long)total;
    h.n_geom = b->n_geom;
    h.chunk = chunk;
    std::memcpy(img.data(), &h, sizeof h);
    std::memcpy(img.data() + a256(sizeof(BatchHeader)), b->entries.data(), b->entries.size() * sizeof(BatchEntry));
    {
        // all entries by population, larger first (ties in table order)
        std::vector<int> ord(b->entries.size());
        for (size_t k = 0; k < ord.size(); ++k) ord[k] = int(k);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return b->entries[a].n > b->entries[c].n; });
        std::vector<EvOrder> evo(ord.size());
        long long acc = 0;
        for (size_t k = 0; k < ord.size(); ++k) {
            evo[k].part_first = acc;
            evo[k].entry = ord[k];
            evo[k].pad = 0;
            acc += b->entries[ord[k]].n;
        }
        if (!evo.empty()) std::memcpy(img.data() + evo_offset(b->n_geom), evo.data(), evo.size() * sizeof(EvOrder));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dev_work, img.data(), img.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "batch_upload: %s", cudaGetErrorString(e)));
    b->chunk = chunk;
    b->uploaded = true;
    b->work = dev_work;
    b->work_bytes = work_bytes;
    return TRK_OK;
}

trk_status run_batched(trk_batch_t b, void* dev_work, const trk_run_opts* opts, void* stream) {
    if (!valid_batch(b) || !dev_work) return trk_status(set_error(TRK_E_INVALID, "run_batched: bad arguments"));
    if (!b->uploaded || b->work != dev_work)
        return trk_status(set_error(TRK_E_INVALID, "run_batched: call batch_upload with this work buffer first"));
    trk_run_opts o;
    trk_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != TRK_FP64 && o.precision != TRK_FP32_LOCAL)
        return trk_status(set_error(TRK_E_INVALID, "run_batched: unknown precision"));
#ifdef TRK_EXACT
    const bool have_f32 = false;
#else
    const bool have_f32 = true;
#endif
    const bool f32 = o.precision == TRK_FP32_LOCAL;
    if (f32 && !have_f32) return trk_status(set_error(TRK_E_UNSUPPORTED, "run_batched: FP32-local is not in the exact build"));
    RunP rp;
    rp.first_id = o.first_id;
    rp.max_segments = o.max_segments ? o.max_segments : 1000000ULL;
    rp.p_absorb = o.p_absorb;
    rp.max_path = DINF;
    rp.seed_lo = uint32_t(o.seed);
    rp.trace_cap = 0;
    rp.mesh = nullptr;
    if (o.mesh_tally) return trk_status(set_error(TRK_E_UNSUPPORTED, "run_batched: no mesh tally in batched mode"));
    bool rec = false;
    for (auto& e : b->entries) rec |= e.records != nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchHeader* hdr = static_cast<BatchHeader*>(dev_work);
    const BatchEntry* table = reinterpret_cast<const BatchEntry*>(static_cast<unsigned char*>(dev_work) + a256(sizeof(BatchHeader)));
    if (o.mode == TRK_MODE_EVENT) return run_batched_event(b, dev_work, o, rp, f32, rec, s);
    if (o.mode != TRK_MODE_HISTORY) return trk_status(set_error(TRK_E_INVALID, "run_batched: unknown mode %d", o.mode));
    const int block = o.block > 0 ? o.block : 128;
    if (block > 128 || (block & 31)) return trk_status(set_error(TRK_E_INVALID, "run_batched: block must be a multiple of 32, <= 128"));
    cudaError_t e = cudaMemsetAsync(&hdr->next_chunk, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_batched: %s", cudaGetErrorString(e)));
    int per_sm = 1;
    int grid = o.grid;
    auto launch = [&](auto kernel) {
        if (grid <= 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
            grid = sm_count_b() * per_sm;
        }
        kernel<<<grid, block, 0, s>>>(hdr, table, rp);
    };
    if (f32) {
#ifndef TRK_EXACT
        if (rec) launch(k_batched<true, F_REC>);
        else launch(k_batched<true, 0>);
#endif
    } else {
        if (rec) launch(k_batched<false, F_REC>);
        else launch(k_batched<false, 0>);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "run_batched: %s", cudaGetErrorString(e)));
    return TRK_OK;
}

// Autotuner: times every (block, chunk) candidate (history mode) or every
// (queue depth, chunk) candidate (event mode) on the batch itself with CUDA
// events (one warm-up and `reps` timed launches each) and returns the fastest
// in opts->block or opts->queue_depth and *chunk_out; the table is left
// uploaded for the winner.  The launches add to the caller's tallies and counters: clear
// them afterwards.  Synchronises `stream`.
trk_status batch_autotune(trk_batch_t b, void* dev_work, size_t work_bytes, trk_run_opts* opts, int* chunk_out,
                          int reps, double* best_ms, void* stream) {
    if (!valid_batch(b) || !dev_work || !opts || !chunk_out) return trk_status(set_error(TRK_E_INVALID, "batch_autotune: bad arguments"));
    if (reps <= 0) reps = 2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // history mode: (block, chunk); event mode: (queue depth, chunk, sort
    // interval).  Event warps keep to one entry's chunks, so small chunks
    // cost no drains and even out the warps' last chunks: on the
    // 64-geometry batch 256 and 512 measured best, 13% ahead of 2048.
    const bool event = opts->mode == TRK_MODE_EVENT;
    const int hist_blocks[] = {64, 96, 128}, hist_chunks[] = {128, 512, 2048};
    const int ev_depths[] = {384, 512}, ev_chunks[] = {128, 256, 512, 2048};
    const int sort_intervals[] = {0, 4};
    const int* blocks = event ? ev_depths : hist_blocks;
    const int* chunks = event ? ev_chunks : hist_chunks;
    const int n_blocks = event ? 2 : 3, n_chunks = event ? 4 : 3;
    const int n_sort = event ? 2 : 1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return trk_status(set_error(TRK_E_CUDA, "batch_autotune: cudaEventCreate failed"));
    float best = 1e30f;
    int best_block = event ? 512 : 128, best_chunk = event ? 512 : 512, best_sort = 0;
    trk_status st = TRK_OK;
    for (int ci = 0; ci < n_chunks && st == TRK_OK; ++ci) {
        const int ch = chunks[ci];
        st = batch_upload(b, dev_work, work_bytes, ch, stream);
        if (st != TRK_OK) break;
        for (int bi = 0; bi < n_blocks && st == TRK_OK; ++bi) {
            for (int si = 0; si < n_sort; ++si) {
                const int bl = blocks[bi];
                trk_run_opts o = *opts;
                if (event) { o.queue_depth = bl; o.sort_interval = sort_intervals[si]; }
                else o.block = bl;
                o.grid = 0;
                st = run_batched(b, dev_work, &o, stream);
                if (st != TRK_OK) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps; ++r) {
                    st = run_batched(b, dev_work, &o, stream);
                    if (st != TRK_OK) break;
                }
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = trk_status(set_error(TRK_E_CUDA, "batch_autotune: sync failed"));
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= float(reps);
                if (ms < best) { best = ms; best_block = bl; best_chunk = ch; best_sort = o.sort_interval; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TRK_OK) return st;
    st = batch_upload(b, dev_work, work_bytes, best_chunk, stream);
    if (st != TRK_OK) return st;
    if (event) { opts->queue_depth = best_block; opts->sort_interval = best_sort; }
    else opts->block = best_block;
    opts->grid = 0;
    *chunk_out = best_chunk;
    if (best_ms) *best_ms = double(best);
    return TRK_OK;
}

}  // extern "C"
