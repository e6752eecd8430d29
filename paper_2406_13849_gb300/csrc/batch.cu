// batch.cu - many independent geometries and particle populations in one
// persistent launch (sm_103a), plus the autotuner that picks its launch shape.
//
// Paper: the tracking loop of Alg. 2 run over many problems at once; the
// paper runs one problem per GPU, this is the serving-style form of it.
//
// Design.  The caller's work buffer holds a device table: one entry per
// geometry (its flattened geometry view, particle buffer, tally, counters,
// tracker) and the prefix sums of its particle chunks.  Warps pull chunk
// indices from one global counter; a chunk is `chunk` particles of a single
// geometry, so the geometry and the tracker type are uniform across the warp
// (warp-level dispatch: one branch per chunk, never per particle).  Chunks
// are numbered with every rect-tracker geometry before every CSG one, so
// neighbouring chunks share code.  run_batched issues only a memset and the
// kernel: after batch_upload it can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "trk.h"
#include "trk_device.cuh"
#include "trk_internal.h"

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
    int csg;
    int pad;
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

}  // namespace

// Host object behind trk_batch_t.
struct trk_batch {
    std::vector<BatchEntry> entries;   // in chunk order (rect trackers first)
    std::vector<int> order;            // entries[k] is input geometry order[k]
    int n_geom = 0;
    int chunk = 0;                     // chunk size the uploaded table was built for
    bool uploaded = false;
    void* work = nullptr;
    unsigned magic = 0;
};
constexpr unsigned TRK_BATCH_MAGIC = 0x74726b62u;

namespace {

bool valid_batch(trk_batch_t b) { return b && b->magic == TRK_BATCH_MAGIC; }

int sm_count_b() {
    int dev = 0, v = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
}

size_t table_bytes(int n) { return a256(sizeof(BatchHeader)) + a256(size_t(n) * sizeof(BatchEntry)); }

}  // namespace

extern "C" {

trk_status batch_create(const trk_geom_t* geoms, int n_geom, const void* const* dev_particles,
                        const int64_t* counts, uint64_t* const* dev_tallies, uint64_t* dev_counters,
                        uint64_t* const* dev_records, int tracker, trk_batch_t* out) {
    if (!geoms || n_geom <= 0 || !dev_particles || !counts || !dev_tallies || !dev_counters || !out)
        return trk_status(set_error(TRK_E_INVALID, "batch_create: null argument or n_geom <= 0"));
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
            return trk_status(set_error(TRK_E_UNSUPPORTED, "batch_create: entry %d has hex arrays (no rect tracker)", k));
        }
        idx[size_t(k)] = k;
    }
    auto use_csg = [&](int k) {
        if (tracker == TRK_TRACKER_CSG) return true;
        return !geoms[k]->rect_ok;
    };
    // rect-tracker geometries first, larger populations first within a type
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
        b->entries.push_back(e);
        b->order.push_back(k);
    }
    b->n_geom = n_geom;
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
    *bytes = table_bytes(b->n_geom);
    return TRK_OK;
}

trk_status batch_upload(trk_batch_t b, void* dev_work, size_t work_bytes, int chunk, void* stream) {
    if (!valid_batch(b) || !dev_work) return trk_status(set_error(TRK_E_INVALID, "batch_upload: bad arguments"));
    if (work_bytes < table_bytes(b->n_geom)) return trk_status(set_error(TRK_E_NOMEM, "batch_upload: work buffer too small"));
    if ((reinterpret_cast<uintptr_t>(dev_work) & 255) != 0)
        return trk_status(set_error(TRK_E_INVALID, "batch_upload: work buffer must be 256-byte aligned"));
    if (chunk <= 0) chunk = 512;
    if (chunk < 32 || chunk > (1 << 20)) return trk_status(set_error(TRK_E_INVALID, "batch_upload: chunk must be in [32, 2^20]"));
    long long total = 0;
    for (auto& e : b->entries) {
        e.first_chunk = total;
        total += (e.n + chunk - 1) / chunk;
    }
    std::vector<unsigned char> img(table_bytes(b->n_geom), 0);
    BatchHeader h;
    h.next_chunk = 0;
    h.total_chunks = (unsigned long long)total;
    h.n_geom = b->n_geom;
    h.chunk = chunk;
    std::memcpy(img.data(), &h, sizeof h);
    std::memcpy(img.data() + a256(sizeof(BatchHeader)), b->entries.data(), b->entries.size() * sizeof(BatchEntry));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dev_work, img.data(), img.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "batch_upload: %s", cudaGetErrorString(e)));
    b->chunk = chunk;
    b->uploaded = true;
    b->work = dev_work;
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
    const int block = o.block > 0 ? o.block : 128;
    if (block > 128 || (block & 31)) return trk_status(set_error(TRK_E_INVALID, "run_batched: block must be a multiple of 32, <= 128"));
    bool rec = false;
    for (auto& e : b->entries) rec |= e.records != nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchHeader* hdr = static_cast<BatchHeader*>(dev_work);
    const BatchEntry* table = reinterpret_cast<const BatchEntry*>(static_cast<unsigned char*>(dev_work) + a256(sizeof(BatchHeader)));
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

// Autotuner: times every (block, chunk) candidate on the batch itself with
// CUDA events (one warm-up and `reps` timed launches each) and returns the
// fastest in opts->block and *chunk_out; the table is left uploaded for the
// winner.  The launches add to the caller's tallies and counters: clear
// them afterwards.  Synchronises `stream`.
trk_status batch_autotune(trk_batch_t b, void* dev_work, size_t work_bytes, trk_run_opts* opts, int* chunk_out,
                          int reps, double* best_ms, void* stream) {
    if (!valid_batch(b) || !dev_work || !opts || !chunk_out) return trk_status(set_error(TRK_E_INVALID, "batch_autotune: bad arguments"));
    if (reps <= 0) reps = 2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks[] = {64, 96, 128};
    const int chunks[] = {128, 512, 2048};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return trk_status(set_error(TRK_E_CUDA, "batch_autotune: cudaEventCreate failed"));
    float best = 1e30f;
    int best_block = 128, best_chunk = 512;
    trk_status st = TRK_OK;
    for (int ch : chunks) {
        st = batch_upload(b, dev_work, work_bytes, ch, stream);
        if (st != TRK_OK) break;
        for (int bl : blocks) {
            trk_run_opts o = *opts;
            o.block = bl;
            o.grid = 0;
            st = run_batched(b, dev_work, &o, stream);
            if (st != TRK_OK) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r) {
                st = run_batched(b, dev_work, &o, stream);
                if (st != TRK_OK) break;
            }
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = trk_status(set_error(TRK_E_CUDA, "batch_autotune: sync failed")); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= float(reps);
            if (ms < best) { best = ms; best_block = bl; best_chunk = ch; }
        }
        if (st != TRK_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TRK_OK) return st;
    st = batch_upload(b, dev_work, work_bytes, best_chunk, stream);
    if (st != TRK_OK) return st;
    opts->block = best_block;
    opts->grid = 0;
    *chunk_out = best_chunk;
    if (best_ms) *best_ms = double(best);
    return TRK_OK;
}

}  // extern "C"
