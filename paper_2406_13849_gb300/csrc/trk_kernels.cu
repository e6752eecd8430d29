// trk_kernels.cu - history-based kernels of the nested-geometry tracker and
// the C-ABI entry points that launch them (sm_103a).
//
// Paper: arXiv 2406.13849.  Alg. 2 (run_histories) with Table 1's tracking
// operations; Alg. 7-10 (multi-universe walk, RTK-style static dispatch);
// Sec. 4.3 (single CSG tracker over pseudo-arrays with a BVH).
//
// Design (GB300):
//  - one thread per history, persistent grid sized from the SM count;
//  - the level stack lives in registers (every loop over levels unrolled to
//    MAXL with runtime guards);
//  - static dispatch per level (the SP idea of Listings 1-4): the rect
//    tracker is compiled in or out by a template flag, never a virtual call;
//  - tallies: one 64-bit integer atomic per segment (order-independent);
//    counters: per-thread registers, warp-reduced, one atomic per warp.
// Built twice: --fmad=false (TRK_EXACT, bit-exact against the FP64 oracle)
// and with contraction (fast).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "trk.h"
// In the history kernel (one history per lane, every step inline) an out-of-
// line find_cell measured faster: 1.33x for the rect tracker, 1.06x for CSG.
#ifndef TRK_FIND_INLINE
#define TRK_FIND_INLINE __noinline__
#endif
#include "trk_device.cuh"
#include "trk_internal.h"
#include "trk_launch.h"

using namespace trk;
using namespace trk::dev;

// Minimum resident 128-thread CTAs per SM the history kernel's register
// allocation must allow (0: let the compiler choose).  Four CTAs (128
// registers a thread) beat the compiler's own choice of ~170 registers.
#ifndef TRK_HIST_MINB
#define TRK_HIST_MINB 4
#endif
#if TRK_HIST_MINB > 0
#define TRK_HIST_BOUNDS __launch_bounds__(128, TRK_HIST_MINB)
#else
#define TRK_HIST_BOUNDS __launch_bounds__(128)
#endif

namespace {


// One history (Alg. 2): flight, then cross or collide, until it ends.
// TK: tracker kind (TK_RECT, TK_CSG, TK_DP).
template <int TK, bool F32, int FLAGS>
__device__ __forceinline__ void history(const DevGeom& g, const ParticlesView& P, long long i, const RunP& rp,
                                        unsigned long long* __restrict__ tally, Counts& cnt,
                                        unsigned long long* __restrict__ rec, int* __restrict__ tr_inst,
                                        double* __restrict__ tr_len) {
    Ctx c;
    c.pid = uint32_t(rp.first_id + uint64_t(i));
    c.event = 0; c.nseg = 0; c.path = 0.0; c.hash = FNV0; c.status = 0;
    int nfis = 0;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    const int pst = P.status[i];
    if (pst != 0) {
        c.status = pst;
        cnt.k[TRK_K_SOURCE]++;
    } else {
        St s;
        load_birth(g, P, i, s);
        if (find_from<TK>(g, s, 0) != 0) {
            c.status = TRK_E_LOST;
            cnt.k[TRK_K_LOST]++;
        } else {
            for (;;) {
                Hit h;
                int a = step_fly<TK, F32, FLAGS>(g, s, h, c, rp, tally, cnt, tr_inst, tr_len, i);
                if (a == A_DONE) break;
                a = (a == A_CROSS) ? step_cross<TK>(g, s, h, c, rp, cnt) : step_collide(g, s, c, rp, cnt);
                if (a == A_DONE) break;
            }
            if ((FLAGS & F_FISS) && c.status == TRK_P_ABSORBED) {
                nfis = fission_sites(g, c.pid, c.event, s.mat, rp);
                fx = s.x; fy = s.y; fz = s.z;
            }
        }
    }
    if (FLAGS & F_FISS) fission_out(rp, i, nfis, fx, fy, fz);
    if (FLAGS & F_REC) {
        rec[2 * i] = c.hash;
        rec[2 * i + 1] = (uint64_t(c.nseg) << 32) | uint32_t(c.status);
    }
    if (FLAGS & F_TRACE) {
        for (long long k = c.nseg; k < rp.trace_cap; ++k) { tr_inst[i * rp.trace_cap + k] = -1; tr_len[i * rp.trace_cap + k] = 0.0; }
    }
}

template <int TK, bool F32, int FLAGS>
__global__ void TRK_HIST_BOUNDS k_history(const DevGeom g, const ParticlesView P, long long n, const RunP rp,
                                                 unsigned long long* __restrict__ tally,
                                                 unsigned long long* __restrict__ counters,
                                                 unsigned long long* __restrict__ rec, int* __restrict__ tr_inst,
                                                 double* __restrict__ tr_len) {
    Counts c;
#pragma unroll
    for (int k = 0; k < NCOUNT; ++k) c.k[k] = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        history<TK, F32, FLAGS>(g, P, i, rp, tally, c, rec, tr_inst, tr_len);
    flush_counts(c, counters);
}

// Builds the DP tracker objects in the geometry's DP region (one thread:
// placement new gives them this module's device virtual tables).
__global__ void k_dp_init(DpTable* t) {
    t->t[0] = new (t->rect) RectTracker();
    t->t[1] = new (t->csg) CsgTracker();
}

// ---------------------------------------------------------------------------
// Birth states (Alg. 2 sampling)
// ---------------------------------------------------------------------------
__device__ bool inside_root(const DevGeom& g, double x, double y, double z) {
    const int4 ui = __ldg(g.u_info + g.root);
    const Pt p = make_pt(x, y, z);
    if (ui.w >= 0) {
        const int4 dm = __ldg(g.l_dim + ui.w), of = __ldg(g.l_off + ui.w);
        return rect_index(g.l_gkey + of.x, dm.x, p.kx, true) >= 0 && rect_index(g.l_gkey + of.y, dm.y, p.ky, true) >= 0 &&
               rect_index(g.l_gkey + of.z, dm.z, p.kz, true) >= 0;
    }
    return csg_search(g, g.root, p, -1, -1, 0) >= 0;
}

__global__ void __launch_bounds__(128) k_source(const DevGeom g, long long n, uint64_t first_id, uint32_t seed_lo,
                                                double* __restrict__ buf) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const uint32_t gid = uint32_t(g.gid);
    double ex[3];
    for (int d = 0; d < 3; ++d) ex[d] = g.src_hi[d] - g.src_lo[d];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t pid = uint32_t(first_id + uint64_t(i));
        double x = 0, y = 0, z = 0, u = 0, v = 0, w = 1, tau = 0;
        int st = TRK_E_SOURCE;
        for (uint32_t a = 0; a < 1000000u; ++a) {
            double xx, xy, xz, unused;
            uniform2(pid, 0, TAG_POSITION, 2 * a, seed_lo, gid, xx, xy);
            uniform2(pid, 0, TAG_POSITION, 2 * a + 1, seed_lo, gid, xz, unused);
            x = g.src_lo[0] + xx * ex[0];
            y = g.src_lo[1] + xy * ex[1];
            z = g.src_lo[2] + xz * ex[2];
            if (inside_root(g, x, y, z)) { st = 0; break; }
        }
        if (st == 0) {
            if (isotropic(pid, 0, seed_lo, gid, u, v, w)) {
                double unused, xt;
                uniform2(pid, 0, TAG_SCALARS, 0, seed_lo, gid, unused, xt);
                tau = -own_log(xt);
            } else {
                st = TRK_E_SOURCE;
            }
        }
        buf[i] = x; buf[n + i] = y; buf[2 * n + i] = z;
        buf[3 * n + i] = u; buf[4 * n + i] = v; buf[5 * n + i] = w;
        buf[6 * n + i] = tau;
        reinterpret_cast<int*>(buf + 7 * n)[i] = st;
    }
}

// ---------------------------------------------------------------------------
// find_cell for points (diagnostic)
// ---------------------------------------------------------------------------
template <bool CSG>
__global__ void __launch_bounds__(128) k_find(const DevGeom g, long long n, const double* __restrict__ xyz,
                                              int64_t* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        St s;
        clear_levels(s);
        s.x = xyz[3 * i]; s.y = xyz[3 * i + 1]; s.z = xyz[3 * i + 2];
        s.lv[0].u = g.root;
        out[i] = find_from<CSG>(g, s, 0) == 0 ? int64_t(instance(s)) : int64_t(-1);
    }
}

// distance_to_surface for points (diagnostic): find_cell from the root, then
// the distance over the levels with the tracking kernels' tie rules.  F32:
// the FP32-local flight's distance (FP32 in the level frames, plane
// crossings re-evaluated in FP64, a close call or an ill-conditioned
// cylinder redone by the FP64 scan; close[i] = 1 then).
template <int TK, bool F32>
__global__ void __launch_bounds__(128) k_distance(const DevGeom g, long long n, const double* __restrict__ xyz,
                                                  const double* __restrict__ dir, double* __restrict__ dist,
                                                  int32_t* __restrict__ level, int64_t* __restrict__ inst,
                                                  int32_t* __restrict__ close) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        St s;
        clear_levels(s);
        s.x = xyz[3 * i]; s.y = xyz[3 * i + 1]; s.z = xyz[3 * i + 2];
        s.d.u = dir[3 * i]; s.d.v = dir[3 * i + 1]; s.d.w = dir[3 * i + 2];
        set_inverse(s.d);
        s.tau = 0.0;
        s.lv[0].u = g.root;
        double d = __longlong_as_double(0x7ff8000000000000LL);
        int lev = -1, cc = 0;
        long long in = -1;
        if (find_from<TK>(g, s, 0) == 0) {
            bool redo = true;
            if constexpr (F32) {
                const DirF df = dir_f32(s.d);
                const Best2 b = distance_f32<TK == TK_CSG>(g, s, df);
                if (!(b.ill || close_call(b.d1, b.d2)) && b.d1 < FINF) {
                    bool exact;
                    d = f32_crossing_length(g, s, b, exact);
                    lev = b.h.level;
                    redo = false;
                } else {
                    cc = 1;
                }
            }
            if (redo) {
                const Hit h = distance_to_boundary<TK>(g, s);
                d = h.d;
                lev = h.level;
            }
            in = instance(s);
        }
        dist[i] = d;
        if (level) level[i] = lev;
        if (inst) inst[i] = in;
        if (close) close[i] = cc;
    }
}

// ---------------------------------------------------------------------------
// Transmission along rays (no collisions) and its backward pass.
// ---------------------------------------------------------------------------
constexpr int NGP = TRK_NGEOM_PARAMS;

// dt/dtheta at the crossing of surface h (position already on it):
// -(df/dtheta) / (grad f . Omega).  Planes tagged pscale sit at G = k pitch
// in the global frame; cylinders tagged rparam j have df/dr_j = -2 r_j and,
// tagged pscale, a centre C = k pitch (df/dpitch = -2 q.C / pitch).
template <bool CSG>
__device__ __forceinline__ void hit_derivative(const DevGeom& g, const St& s, const Hit& h, double pitch,
                                               double dt[NGP]) {
#pragma unroll
    for (int j = 0; j < NGP; ++j) dt[j] = 0.0;
    double Tx = 0.0, Ty = 0.0;
#pragma unroll
    for (int l = 0; l < MAXL; ++l)
        if (l < h.level) { Tx += s.lv[l].tx; Ty += s.lv[l].ty; }
    if (h.surf < 0) {
        // rect array plane (rect view)
        int lat = -1, idx = 0;
#pragma unroll
        for (int l = 0; l < MAXL; ++l)
            if (l == h.level) {
                lat = __ldg(g.u_info + s.lv[l].u).w;
                idx = h.dim == 0 ? s.lv[l].i : (h.dim == 1 ? s.lv[l].j : s.lv[l].k);
            }
        if (lat < 0 || h.dim > 1 || !__ldg(g.l_pscale + lat) || !(pitch > 0.0)) return;
        const int4 of = __ldg(g.l_off + lat);
        const int go = h.dim == 0 ? of.x : of.y;
        const double G = __ldg(g.l_grid + go + idx + (h.dsign > 0)) + (h.dim == 0 ? Tx : Ty);
        dt[3] = (G / pitch) / (h.dim == 0 ? s.d.u : s.d.v);
        return;
    }
    const int info = __ldg(g.s_info + h.surf);
    const int type = info & 15, rparam = ((info >> 8) & 15) - 1, pscale = (info >> 12) & 1;
    double c0, c1, c2, c3;
    load_coef(g, h.surf, c0, c1, c2, c3);
    if (type == S_PX || type == S_PY) {
        if (pscale && pitch > 0.0) {
            const double G = c0 + (type == S_PX ? Tx : Ty);
            dt[3] = (G / pitch) / (type == S_PX ? s.d.u : s.d.v);
        }
    } else if (type == S_CZ) {
        const double cx = c0 + Tx, cy = c1 + Ty;
        const double qx = s.x - cx, qy = s.y - cy;
        const double gd = 2.0 * (qx * s.d.u + qy * s.d.v);
        if (gd == 0.0) return;
        if (rparam >= 0 && rparam < 3) {
            const double v = -(-2.0 * c2) / gd;
            if (rparam == 0) dt[0] = v;
            else if (rparam == 1) dt[1] = v;
            else dt[2] = v;
        }
        if (pscale && pitch > 0.0) dt[3] = -(-2.0 * (qx * cx + qy * cy) / pitch) / gd;
    }
}

// One ray's walk as a resumable state: the tracker state, per-material
// lengths and, for BWD, the sigma-weighted derivative of the optical depth
// with respect to theta (din: the derivative of the current segment's entry
// point).  ray_start places the ray (find_cell); ray_step walks one segment
// and returns false once the ray has left the geometry or ended otherwise.
struct RayWalk {
    St s;
    double lens[MAXMAT], dtau[NGP], din[NGP];
    int nseg;
};

template <bool CSG>
__device__ __forceinline__ bool ray_start(const DevGeom& g, const double* ray, RayWalk& r) {
#pragma unroll
    for (int m = 0; m < MAXMAT; ++m) r.lens[m] = 0.0;
#pragma unroll
    for (int j = 0; j < NGP; ++j) { r.dtau[j] = 0.0; r.din[j] = 0.0; }
    r.nseg = 0;
    clear_levels(r.s);
    r.s.x = ray[0]; r.s.y = ray[1]; r.s.z = ray[2];
    r.s.d.u = ray[3]; r.s.d.v = ray[4]; r.s.d.w = ray[5];
    r.s.tau = 0.0;
    set_inverse(r.s.d);
    r.s.lv[0].u = g.root;
    return find_from<CSG>(g, r.s, 0) == 0;
}

template <bool CSG, bool BWD>
__device__ __forceinline__ bool ray_step(const DevGeom& g, const double* sigma, double pitch, RayWalk& r) {
    St& s = r.s;
    if (r.nseg >= 10000000) return false;
    ++r.nseg;
    const Hit h = distance_to_boundary<CSG>(g, s);
    if (!d_finite_lt_inf(h.d)) return false;
    const int m = s.mat;
#pragma unroll
    for (int k = 0; k < MAXMAT; ++k)
        if (k == m) r.lens[k] += h.d;
    s.x = s.x + h.d * s.d.u;
    s.y = s.y + h.d * s.d.v;
    s.z = s.z + h.d * s.d.w;
    if (BWD) {
        double dout[NGP];
        hit_derivative<CSG>(g, s, h, pitch, dout);
        const double sg = __ldg(sigma + m);
#pragma unroll
        for (int j = 0; j < NGP; ++j) { r.dtau[j] += sg * (dout[j] - r.din[j]); r.din[j] = dout[j]; }
    }
    int fl;
    int cr = cross_surface<CSG>(g, s, h, fl);
    if (cr == CR_FIND) cr = find_from<CSG>(g, s, fl) == 0 ? CR_OK : CR_LOST;
    return cr != CR_ESCAPE && cr != CR_LOST;
}

// Rays per thread: each thread walks a fixed list of RAYS_PER_THREAD rays as
// one loop (a lane whose ray ends starts its next one at once), so the lanes
// of a warp stay busy until their lists run out instead of waiting for the
// warp's longest ray; the lists are fixed, so the order of every sum is too.
// Block b holds rays [b * RAY_TILE, (b + 1) * RAY_TILE), its thread t the
// rays b * RAY_TILE + t + k * RAY_BLOCK, k < RAYS_PER_THREAD.
constexpr int RAY_BLOCK = 128;
constexpr int RAYS_PER_THREAD = 8;
constexpr long long RAY_TILE = (long long)RAY_BLOCK * RAYS_PER_THREAD;
static_assert(RAY_TILE == TRK_RAYS_PER_BLOCK, "the work-buffer layout assumes this tile");

template <bool CSG>
__global__ void __launch_bounds__(RAY_BLOCK) k_transmission(const DevGeom g, long long n, const double* __restrict__ rays,
                                                            const double* __restrict__ sigma, double* __restrict__ T,
                                                            double* __restrict__ lens_out) {
    const int nm = g.n_mat;
    const long long base = (long long)blockIdx.x * RAY_TILE + threadIdx.x;
    int k = 0;
    long long i = base;
    bool have = i < n;
    RayWalk r;
    bool live = have && ray_start<CSG>(g, rays + 6 * i, r);
    while (have) {
        if (live) live = ray_step<CSG, false>(g, sigma, 0.0, r);
        if (live) continue;
        double opt = 0.0;
#pragma unroll
        for (int m = 0; m < MAXMAT; ++m)
            if (m < nm) opt += __ldg(sigma + m) * r.lens[m];
        T[i] = exp(-opt);
        if (lens_out) {
#pragma unroll
            for (int m = 0; m < MAXMAT; ++m)
                if (m < nm) lens_out[i * nm + m] = r.lens[m];
        }
        ++k;
        i = base + (long long)k * RAY_BLOCK;
        have = k < RAYS_PER_THREAD && i < n;
        live = have && ray_start<CSG>(g, rays + 6 * i, r);
    }
}

// Per block: the sum over its rays of gT * dT/dtheta into
// partial[block][nm + NGP] (each thread adds its rays in list order, then a
// fixed tree over the block's threads); a second kernel adds the partials in
// block order.
template <bool CSG>
__global__ void __launch_bounds__(RAY_BLOCK) k_transmission_bwd(const DevGeom g, long long n,
                                                                const double* __restrict__ rays,
                                                                const double* __restrict__ sigma, double pitch,
                                                                const double* __restrict__ gT,
                                                                double* __restrict__ partial) {
    const int nm = g.n_mat;
    const int nq = nm + NGP;
    __shared__ double red[RAY_BLOCK];
    double acc[MAXMAT + NGP];
#pragma unroll
    for (int j = 0; j < MAXMAT + NGP; ++j) acc[j] = 0.0;
    const long long base = (long long)blockIdx.x * RAY_TILE + threadIdx.x;
    int k = 0;
    long long i = base;
    bool have = i < n;
    RayWalk r;
    bool live = have && ray_start<CSG>(g, rays + 6 * i, r);
    while (have) {
        if (live) live = ray_step<CSG, true>(g, sigma, pitch, r);
        if (live) continue;
        double opt = 0.0;
#pragma unroll
        for (int m = 0; m < MAXMAT; ++m)
            if (m < nm) opt += __ldg(sigma + m) * r.lens[m];
        const double Tv = exp(-opt);
        const double gi = gT[i];
#pragma unroll
        for (int m = 0; m < MAXMAT; ++m)
            if (m < nm) acc[m] += gi * (-r.lens[m] * Tv);
#pragma unroll
        for (int j = 0; j < NGP; ++j) acc[MAXMAT + j] += gi * (-Tv * r.dtau[j]);
        ++k;
        i = base + (long long)k * RAY_BLOCK;
        have = k < RAYS_PER_THREAD && i < n;
        live = have && ray_start<CSG>(g, rays + 6 * i, r);
    }
    for (int q = 0; q < nq; ++q) {
        const int slot = q < nm ? q : MAXMAT + (q - nm);
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < MAXMAT + NGP; ++j)
            if (j == slot) v = acc[j];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int w = RAY_BLOCK / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * nq + q] = red[0];
        __syncthreads();
    }
}

__global__ void k_reduce_partials(const double* __restrict__ partial, long long nblocks, int nq,
                                  double* __restrict__ out) {
    const int q = threadIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (long long b = 0; b < nblocks; ++b) s += partial[b * nq + q];
    out[q] = s;
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

template <class K>
int persistent_grid(K kernel, int block, long long n, int requested) {
    if (requested > 0) return requested;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    long long want = (n + block - 1) / block;
    long long full = (long long)sm_count() * per_sm;
    if (want < 1) want = 1;
    return int(want < full ? want : full);
}

bool valid(trk_geom_t g) { return g && g->magic == TRK_GEOM_MAGIC; }

ParticlesView view_of(const void* dev_particles, long long n) {
    const double* b = static_cast<const double*>(dev_particles);
    ParticlesView p;
    p.x = b; p.y = b + n; p.z = b + 2 * n; p.u = b + 3 * n; p.v = b + 4 * n; p.w = b + 5 * n; p.tau = b + 6 * n;
    p.status = reinterpret_cast<const int*>(b + 7 * n);
    return p;
}

size_t particle_bytes(long long n) { return size_t(n) * (7 * sizeof(double) + sizeof(int)); }

trk_status launch_error(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "%s: %s", where, cudaGetErrorString(e)));
    return TRK_OK;
}

int resolve_tracker(trk_geom_t g, int tracker, trk_status* st, bool allow_dp = false, bool event = false) {
    *st = TRK_OK;
    if (tracker == TRK_TRACKER_DP && allow_dp) return tracker;
    // AUTO: the array tracker for the history kernels, except for geometries
    // with hex arrays, where the BVH-CSG tracker measured as fast or faster
    // (its BVH walk and the closed-form hex search cost about the same; the
    // CSG kernels are smaller).  The event kernels take the CSG tracker
    // everywhere: its kernel is the smaller (slab cells stand in for the
    // array levels) and measured 1.25x the array tracker's on the 15 x 15
    // assembly core.  Both trackers give the same histories bit for bit.
    if (tracker == TRK_TRACKER_AUTO)
        return (g->rect_ok && !g->has_hex && !event) ? TRK_TRACKER_RECT : TRK_TRACKER_CSG;
    if (tracker == TRK_TRACKER_RECT && !g->rect_ok) {
        *st = trk_status(set_error(TRK_E_UNSUPPORTED, "array tracker not available for this geometry"));
        return -1;
    }
    if (tracker != TRK_TRACKER_RECT && tracker != TRK_TRACKER_CSG) {
        *st = trk_status(set_error(TRK_E_INVALID, "unknown tracker %d", tracker));
        return -1;
    }
    return tracker;
}

template <int TK, bool F32, int FLAGS>
trk_status launch_history(trk_geom_t g, const ParticlesView& P, long long n, const RunP& rp,
                          unsigned long long* tally, unsigned long long* cnt, unsigned long long* rec, int* ti,
                          double* tl, int block, int grid, cudaStream_t s) {
    auto k = k_history<TK, F32, FLAGS>;
    const int gr = persistent_grid(k, block, n, grid);
    k<<<gr, block, 0, s>>>(g->dg, P, n, rp, tally, cnt, rec, ti, tl);
    return launch_error("run_histories");
}

// The FP32-local kernels exist in the fast build only (the exact build is
// the path that is bit-exact against the FP64 oracle).
#ifdef TRK_EXACT
constexpr bool HAVE_F32 = false;
#else
constexpr bool HAVE_F32 = true;
#endif

}  // namespace

int trk::dp_install(void* dev, void* stream) {
    k_dp_init<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<DpTable*>(dev));
    return int(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

int trk_exact_build(void) {
#ifdef TRK_EXACT
    return 1;
#else
    return 0;
#endif
}

trk_status source_init(trk_geom_t g, int64_t n, uint64_t first_id, uint64_t seed, void* dev_particles,
                       size_t* bytes, void* stream) {
    if (!valid(g) || !bytes) return trk_status(set_error(TRK_E_INVALID, "source_init: invalid handle or bytes"));
    if (n < 0) return trk_status(set_error(TRK_E_INVALID, "source_init: n < 0"));
    const size_t need = particle_bytes(n);
    if (!dev_particles) { *bytes = need; return TRK_OK; }
    if (*bytes < need) { *bytes = need; return trk_status(set_error(TRK_E_NOMEM, "source_init: buffer too small")); }
    if ((reinterpret_cast<uintptr_t>(dev_particles) & 7) != 0)
        return trk_status(set_error(TRK_E_INVALID, "source_init: buffer must be 8-byte aligned"));
    if (n == 0) return TRK_OK;
    const int block = 128;
    const int grid = persistent_grid(k_source, block, n, 0);
    k_source<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(g->dg, n, first_id, uint32_t(seed),
                                                                      static_cast<double*>(dev_particles));
    return launch_error("source_init");
}

constexpr int DEFAULT_SLOTS = 256;

int event_slots(const trk_run_opts& o) { return o.queue_depth > 0 ? o.queue_depth : DEFAULT_SLOTS; }

trk_status run_histories_work_bytes(trk_geom_t g, int64_t n, const trk_run_opts* opts, size_t* bytes) {
    if (!valid(g) || !bytes || n < 0) return trk_status(set_error(TRK_E_INVALID, "run_histories_work_bytes: bad arguments"));
    trk_run_opts o;
    trk_default_opts(&o);
    if (opts) o = *opts;
    *bytes = 0;
    if (o.mode == TRK_MODE_EVENT) {
        const int slots = event_slots(o);
        if (slots < 32 || slots > 512) return trk_status(set_error(TRK_E_INVALID, "queue_depth must be in [32, 512]"));
        const int grid = o.grid > 0 ? o.grid : event_grid(slots);
        *bytes = event_work_bytes(slots, grid);
    }
    return TRK_OK;
}

trk_status run_histories(trk_geom_t g, const void* dev_particles, int64_t n, uint64_t* dev_tally,
                         uint64_t* dev_counters, uint64_t* dev_records, void* dev_work, size_t work_bytes,
                         const trk_run_opts* opts, void* stream) {
    if (!valid(g)) return trk_status(set_error(TRK_E_INVALID, "run_histories: invalid handle"));
    if (n < 0 || (n > 0 && (!dev_particles || !dev_tally || !dev_counters)))
        return trk_status(set_error(TRK_E_INVALID, "run_histories: null buffer or n < 0"));
    if (n > (int64_t(1) << 32)) return trk_status(set_error(TRK_E_INVALID, "run_histories: n exceeds 2^32 particle ids"));
    trk_run_opts o;
    trk_default_opts(&o);
    if (opts) o = *opts;
    trk_status st;
    const int tracker = resolve_tracker(g, o.tracker, &st, true, o.mode == TRK_MODE_EVENT);
    if (tracker < 0) return st;
    if (o.mode != TRK_MODE_HISTORY && o.mode != TRK_MODE_EVENT)
        return trk_status(set_error(TRK_E_INVALID, "run_histories: unknown mode %d", o.mode));
    if (o.precision != TRK_FP64 && o.precision != TRK_FP32_LOCAL)
        return trk_status(set_error(TRK_E_INVALID, "run_histories: unknown precision %d", o.precision));
    const bool dp = tracker == TRK_TRACKER_DP;
    if (dp && (o.mode != TRK_MODE_HISTORY || o.precision != TRK_FP64 || o.mesh_tally ||
               (o.max_path > 0.0 && o.max_path < DINF)))
        return trk_status(set_error(TRK_E_UNSUPPORTED,
                                    "run_histories: the DP tracker runs the FP64 history kernel without mesh tally or path cutoff"));
    const bool f32 = o.precision == TRK_FP32_LOCAL;
    if (f32 && !HAVE_F32)
        return trk_status(set_error(TRK_E_UNSUPPORTED, "run_histories: FP32-local is not in the exact (--fmad=false) build"));
    if (!(o.p_absorb >= 0.0 && o.p_absorb <= 1.0)) return trk_status(set_error(TRK_E_INVALID, "run_histories: p_absorb outside [0,1]"));
    if (n == 0) return TRK_OK;
    RunP rp;
    rp.first_id = o.first_id;
    rp.max_segments = o.max_segments ? o.max_segments : 1000000ULL;
    rp.p_absorb = o.p_absorb;
    const bool cut = o.max_path > 0.0 && o.max_path < DINF;
    rp.max_path = cut ? o.max_path : DINF;
    rp.seed_lo = uint32_t(o.seed);
    rp.trace_cap = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ParticlesView P = view_of(dev_particles, n);
    auto* T = reinterpret_cast<unsigned long long*>(dev_tally);
    auto* C = reinterpret_cast<unsigned long long*>(dev_counters);
    auto* R = reinterpret_cast<unsigned long long*>(dev_records);
    const bool csg = tracker == TRK_TRACKER_CSG;
    const bool mesh = o.mesh_tally != nullptr;
    rp.mesh = reinterpret_cast<unsigned long long*>(o.mesh_tally);
    const int flags = (dev_records ? F_REC : 0) | (cut ? F_CUT : 0) | (mesh ? F_MESH : 0);
    if (f32 && cut) return trk_status(set_error(TRK_E_UNSUPPORTED, "run_histories: path cutoff needs FP64 precision"));
    if (mesh && !g->dg.m_n[0])
        return trk_status(set_error(TRK_E_INVALID, "run_histories: mesh tally given but the geometry has no mesh"));
    if (mesh && (f32 || cut))
        return trk_status(set_error(TRK_E_UNSUPPORTED, "run_histories: the mesh tally needs FP64 precision and no path cutoff"));
    if (o.mode == TRK_MODE_EVENT) {
        const int slots = event_slots(o);
        if (slots < 32 || slots > 512) return trk_status(set_error(TRK_E_INVALID, "queue_depth must be in [32, 512]"));
        const int grid = o.grid > 0 ? o.grid : event_grid(slots);
        if (o.max_rounds < 0) return trk_status(set_error(TRK_E_INVALID, "max_rounds must be >= 0"));
        if (o.sort_interval < 0) return trk_status(set_error(TRK_E_INVALID, "sort_interval must be >= 0"));
        return launch_event(g, P, n, rp, csg, f32, flags, T, C, R, dev_work, work_bytes, slots, grid, o.max_rounds,
                            o.sort_interval, s);
    }
    const int block = o.block > 0 ? o.block : 128;
    if (block > 128 || (block & 31)) return trk_status(set_error(TRK_E_INVALID, "run_histories: block must be a multiple of 32, <= 128"));
#define TRK_LAUNCH(CSGV, F32V, F) return launch_history<CSGV, F32V, F>(g, P, n, rp, T, C, R, nullptr, nullptr, block, o.grid, s)
    if (dp) {
        if (flags & F_REC) TRK_LAUNCH(TK_DP, false, F_REC);
        TRK_LAUNCH(TK_DP, false, 0);
    }
    if (f32) {
#ifndef TRK_EXACT
        if (csg) {
            if (flags & F_REC) TRK_LAUNCH(true, true, F_REC);
            TRK_LAUNCH(true, true, 0);
        }
        if (flags & F_REC) TRK_LAUNCH(false, true, F_REC);
        TRK_LAUNCH(false, true, 0);
#endif
    }
    if (csg) {
        switch (flags) {
            case 0: TRK_LAUNCH(true, false, 0);
            case F_REC: TRK_LAUNCH(true, false, F_REC);
            case F_CUT: TRK_LAUNCH(true, false, F_CUT);
            case F_MESH: TRK_LAUNCH(true, false, F_MESH);
            case F_MESH | F_REC: TRK_LAUNCH(true, false, F_MESH | F_REC);
            default: TRK_LAUNCH(true, false, F_REC | F_CUT);
        }
    } else {
        switch (flags) {
            case 0: TRK_LAUNCH(false, false, 0);
            case F_REC: TRK_LAUNCH(false, false, F_REC);
            case F_CUT: TRK_LAUNCH(false, false, F_CUT);
            case F_MESH: TRK_LAUNCH(false, false, F_MESH);
            case F_MESH | F_REC: TRK_LAUNCH(false, false, F_MESH | F_REC);
            default: TRK_LAUNCH(false, false, F_REC | F_CUT);
        }
    }
#undef TRK_LAUNCH
}

trk_status trk_trace(trk_geom_t g, const void* dev_particles, int64_t n, int32_t cap, int32_t* dev_inst,
                     double* dev_len, uint64_t* dev_tally, uint64_t* dev_counters, void* dev_work,
                     size_t work_bytes, const trk_run_opts* opts, void* stream) {
    if (!valid(g) || n < 0 || cap <= 0 ||
        (n > 0 && (!dev_particles || !dev_inst || !dev_len || !dev_tally || !dev_counters)))
        return trk_status(set_error(TRK_E_INVALID, "trk_trace: bad arguments"));
    trk_run_opts o;
    trk_default_opts(&o);
    if (opts) o = *opts;
    trk_status st;
    const int tracker = resolve_tracker(g, o.tracker, &st);
    if (tracker < 0) return st;
    if (n == 0) return TRK_OK;
    RunP rp;
    rp.first_id = o.first_id;
    rp.max_segments = o.max_segments ? o.max_segments : 1000000ULL;
    rp.p_absorb = o.p_absorb;
    rp.max_path = DINF;
    rp.seed_lo = uint32_t(o.seed);
    rp.trace_cap = cap;
    rp.mesh = nullptr;
    auto* T = reinterpret_cast<unsigned long long*>(dev_tally);
    auto* C = reinterpret_cast<unsigned long long*>(dev_counters);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ParticlesView P = view_of(dev_particles, n);
    if (o.precision != TRK_FP64 && o.precision != TRK_FP32_LOCAL)
        return trk_status(set_error(TRK_E_INVALID, "trk_trace: unknown precision %d", o.precision));
    if (o.mode == TRK_MODE_EVENT) {
        // the persistent event kernel in the launch shape run_histories uses
        // for these options, with the segment log switched on
        if (o.precision == TRK_FP32_LOCAL && !HAVE_F32)
            return trk_status(set_error(TRK_E_UNSUPPORTED, "trk_trace: FP32-local is not in the exact build"));
        const int slots = event_slots(o);
        if (slots < 32 || slots > 512) return trk_status(set_error(TRK_E_INVALID, "queue_depth must be in [32, 512]"));
        const int grid = o.grid > 0 ? o.grid : event_grid(slots);
        if (o.max_rounds < 0) return trk_status(set_error(TRK_E_INVALID, "max_rounds must be >= 0"));
        rp.tr_inst = dev_inst;
        rp.tr_len = dev_len;
        return launch_event(g, P, n, rp, tracker == TRK_TRACKER_CSG, o.precision == TRK_FP32_LOCAL, F_TRACE, T, C,
                            nullptr, dev_work, work_bytes, slots, grid, o.max_rounds, o.sort_interval, s);
    }
    if (o.mode != TRK_MODE_HISTORY) return trk_status(set_error(TRK_E_INVALID, "trk_trace: unknown mode %d", o.mode));
    if (o.precision == TRK_FP32_LOCAL) {
#ifndef TRK_EXACT
        if (tracker == TRK_TRACKER_CSG)
            return launch_history<true, true, F_TRACE>(g, P, n, rp, T, C, nullptr, dev_inst, dev_len, 128, 0, s);
        return launch_history<false, true, F_TRACE>(g, P, n, rp, T, C, nullptr, dev_inst, dev_len, 128, 0, s);
#else
        return trk_status(set_error(TRK_E_UNSUPPORTED, "trk_trace: FP32-local is not in the exact build"));
#endif
    }
    if (tracker == TRK_TRACKER_CSG)
        return launch_history<true, false, F_TRACE>(g, P, n, rp, T, C, nullptr, dev_inst, dev_len, 128, 0, s);
    return launch_history<false, false, F_TRACE>(g, P, n, rp, T, C, nullptr, dev_inst, dev_len, 128, 0, s);
}

trk_status tally_read(trk_geom_t g, const uint64_t* dev_tally, double* host_out, int64_t n_inst,
                      const uint64_t* dev_counters, void* stream) {
    if (!valid(g) || !dev_tally || !host_out) return trk_status(set_error(TRK_E_INVALID, "tally_read: bad arguments"));
    if (n_inst != g->n_inst) return trk_status(set_error(TRK_E_INVALID, "tally_read: n_instances %lld != %lld", (long long)n_inst, (long long)g->n_inst));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // convert in place on the host: copy the integers into the output array's storage
    static_assert(sizeof(double) == sizeof(uint64_t), "layout");
    cudaError_t e = cudaMemcpyAsync(host_out, dev_tally, size_t(n_inst) * 8, cudaMemcpyDeviceToHost, s);
    uint64_t status = 0;
    if (e == cudaSuccess && dev_counters)
        e = cudaMemcpyAsync(&status, dev_counters + TRK_K_STATUS, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "tally_read: %s", cudaGetErrorString(e)));
    uint64_t* raw = reinterpret_cast<uint64_t*>(host_out);
    for (int64_t i = 0; i < n_inst; ++i) host_out[i] = double(raw[i]) * 0x1.0p-32;
    if (status != 0) return trk_status(set_error(int(int64_t(status)), "tally_read: kernel reported status %lld", (long long)int64_t(status)));
    return TRK_OK;
}

trk_status trk_find_cell(trk_geom_t g, int tracker, int64_t n, const double* dev_xyz, int64_t* dev_inst, void* stream) {
    if (!valid(g) || n < 0 || (n > 0 && (!dev_xyz || !dev_inst))) return trk_status(set_error(TRK_E_INVALID, "trk_find_cell: bad arguments"));
    trk_status st;
    const int t = resolve_tracker(g, tracker, &st);
    if (t < 0) return st;
    if (n == 0) return TRK_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (t == TRK_TRACKER_CSG) {
        const int gr = persistent_grid(k_find<true>, 128, n, 0);
        k_find<true><<<gr, 128, 0, s>>>(g->dg, n, dev_xyz, dev_inst);
    } else {
        const int gr = persistent_grid(k_find<false>, 128, n, 0);
        k_find<false><<<gr, 128, 0, s>>>(g->dg, n, dev_xyz, dev_inst);
    }
    return launch_error("trk_find_cell");
}

trk_status trk_distance_to_surface(trk_geom_t g, int tracker, int precision, int64_t n, const double* dev_xyz,
                                   const double* dev_dir, double* dev_dist, int32_t* dev_level, int64_t* dev_inst,
                                   int32_t* dev_close, void* stream) {
    if (!valid(g) || n < 0 || (n > 0 && (!dev_xyz || !dev_dir || !dev_dist)))
        return trk_status(set_error(TRK_E_INVALID, "trk_distance_to_surface: bad arguments"));
    if (precision != TRK_FP64 && precision != TRK_FP32_LOCAL)
        return trk_status(set_error(TRK_E_INVALID, "trk_distance_to_surface: unknown precision %d", precision));
    trk_status st;
    const int t = resolve_tracker(g, tracker, &st, true);
    if (t < 0) return st;
    const bool f32 = precision == TRK_FP32_LOCAL;
    if (f32 && (!HAVE_F32 || t == TRK_TRACKER_DP))
        return trk_status(set_error(TRK_E_UNSUPPORTED, "trk_distance_to_surface: FP32-local needs the fast build and "
                                                       "the array or CSG tracker"));
    if (n == 0) return TRK_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
#define TRK_DIST(TKV, F32V)                                                                                        \
    do {                                                                                                           \
        const int gr = persistent_grid(k_distance<TKV, F32V>, 128, n, 0);                                          \
        k_distance<TKV, F32V><<<gr, 128, 0, s>>>(g->dg, n, dev_xyz, dev_dir, dev_dist, dev_level, dev_inst,        \
                                                 dev_close);                                                       \
    } while (0)
    if (f32) {
#ifndef TRK_EXACT
        if (t == TRK_TRACKER_CSG) TRK_DIST(TK_CSG, true);
        else TRK_DIST(TK_RECT, true);
#endif
    } else if (t == TRK_TRACKER_CSG) TRK_DIST(TK_CSG, false);
    else if (t == TRK_TRACKER_DP) TRK_DIST(TK_DP, false);
    else TRK_DIST(TK_RECT, false);
#undef TRK_DIST
    return launch_error("trk_distance_to_surface");
}

trk_status trk_sync_status(const uint64_t* dev_counters, void* stream) {
    if (!dev_counters) return trk_status(set_error(TRK_E_INVALID, "trk_sync_status: null counters"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, dev_counters + TRK_K_STATUS, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "trk_sync_status: %s", cudaGetErrorString(e)));
    if (status != 0) return trk_status(set_error(int(int64_t(status)), "kernel reported status %lld", (long long)int64_t(status)));
    return TRK_OK;
}

trk_status transmission_fwd(trk_geom_t g, int tracker, int64_t n, const double* dev_rays, const double* dev_sigma,
                            double* dev_T, double* dev_lens, void* stream) {
    if (!valid(g) || n < 0 || (n > 0 && (!dev_rays || !dev_sigma || !dev_T)))
        return trk_status(set_error(TRK_E_INVALID, "transmission_fwd: bad arguments"));
    if (g->n_mat > MAXMAT) return trk_status(set_error(TRK_E_UNSUPPORTED, "transmission_fwd: more than %d materials", MAXMAT));
    trk_status st;
    const int t = resolve_tracker(g, tracker, &st);
    if (t < 0) return st;
    if (n == 0) return TRK_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nb = (n + RAY_TILE - 1) / RAY_TILE;
    if (t == TRK_TRACKER_CSG)
        k_transmission<true><<<unsigned(nb), RAY_BLOCK, 0, s>>>(g->dg, n, dev_rays, dev_sigma, dev_T, dev_lens);
    else
        k_transmission<false><<<unsigned(nb), RAY_BLOCK, 0, s>>>(g->dg, n, dev_rays, dev_sigma, dev_T, dev_lens);
    return launch_error("transmission_fwd");
}

trk_status transmission_bwd_work_bytes(trk_geom_t g, int64_t n, size_t* bytes) {
    if (!valid(g) || n < 0 || !bytes) return trk_status(set_error(TRK_E_INVALID, "transmission_bwd_work_bytes: bad arguments"));
    const long long nb = (n + RAY_TILE - 1) / RAY_TILE;
    *bytes = size_t(nb > 0 ? nb : 1) * size_t(g->n_mat + NGP) * sizeof(double);
    return TRK_OK;
}

trk_status transmission_bwd(trk_geom_t g, int tracker, int64_t n, const double* dev_rays, const double* dev_sigma,
                            double pitch, const double* dev_gT, double* dev_grad, void* dev_work, size_t work_bytes,
                            void* stream) {
    if (!valid(g) || n < 0 || !dev_grad || (n > 0 && (!dev_rays || !dev_sigma || !dev_gT)))
        return trk_status(set_error(TRK_E_INVALID, "transmission_bwd: bad arguments"));
    if (g->n_mat > MAXMAT) return trk_status(set_error(TRK_E_UNSUPPORTED, "transmission_bwd: more than %d materials", MAXMAT));
    size_t need = 0;
    transmission_bwd_work_bytes(g, n, &need);
    if (!dev_work || work_bytes < need) return trk_status(set_error(TRK_E_NOMEM, "transmission_bwd: work buffer needs %zu bytes", need));
    trk_status st;
    const int t = resolve_tracker(g, tracker, &st);
    if (t < 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nb = (n + RAY_TILE - 1) / RAY_TILE;
    const int nq = g->n_mat + NGP;
    double* partial = static_cast<double*>(dev_work);
    if (nb == 0) {
        cudaMemsetAsync(dev_grad, 0, size_t(nq) * sizeof(double), s);
        return launch_error("transmission_bwd");
    }
    if (t == TRK_TRACKER_CSG)
        k_transmission_bwd<true><<<unsigned(nb), RAY_BLOCK, 0, s>>>(g->dg, n, dev_rays, dev_sigma, pitch, dev_gT, partial);
    else
        k_transmission_bwd<false><<<unsigned(nb), RAY_BLOCK, 0, s>>>(g->dg, n, dev_rays, dev_sigma, pitch, dev_gT, partial);
    trk_status e = launch_error("transmission_bwd");
    if (e != TRK_OK) return e;
    k_reduce_partials<<<1, 32, 0, s>>>(partial, nb, nq, dev_grad);
    return launch_error("transmission_bwd reduce");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Power iteration (Alg. 1): cycles of run_histories whose births come from
// the previous cycle's fission bank.  The bank keeps the sites in history
// order (a block scan of the per-history counts), so the births of the next
// cycle, which pick sites by index, do not depend on thread timing.
// ---------------------------------------------------------------------------
namespace {

constexpr int BANK_BLOCK = 1024;

// Exclusive scan over a block of BANK_BLOCK threads; *total gets the sum.
__device__ long long block_exclusive_scan(long long v, long long* total) {
    __shared__ long long wsum[BANK_BLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    const long long before = w > 0 ? wsum[w - 1] : 0;
    *total = wsum[BANK_BLOCK / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(BANK_BLOCK) k_bank_count(const int* __restrict__ fis_n, long long n,
                                                           long long* __restrict__ bsum) {
    const long long i = (long long)blockIdx.x * BANK_BLOCK + threadIdx.x;
    long long tot;
    block_exclusive_scan(i < n ? fis_n[i] : 0, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block: block sums to offsets, the bank size, and the cycle's
// k = (double(nu sum) * 2^-32) / n, the next cycle's normalisation.
__global__ void __launch_bounds__(BANK_BLOCK) k_bank_scan(long long* __restrict__ bsum, long long nb, long long n,
                                                          const unsigned long long* __restrict__ nu_sum,
                                                          double* __restrict__ knorm, double* __restrict__ k_out,
                                                          long long* __restrict__ bank_out,
                                                          long long* __restrict__ bank_size,
                                                          unsigned long long* __restrict__ counters) {
    long long carry = 0;
    for (long long base = 0; base < nb; base += BANK_BLOCK) {
        const long long idx = base + threadIdx.x;
        const long long v = idx < nb ? bsum[idx] : 0;
        long long tot;
        const long long ex = block_exclusive_scan(v, &tot);
        if (idx < nb) bsum[idx] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *bank_size = carry;
        *bank_out = carry;
        const double k = (double(*nu_sum) * 0x1p-32) / double(n);
        *k_out = k;
        *knorm = k;
        if (carry == 0) kernel_status(counters, TRK_E_SOURCE);
    }
}

__global__ void __launch_bounds__(BANK_BLOCK) k_bank_write(const int* __restrict__ fis_n,
                                                           const double* __restrict__ fis_pos, long long n,
                                                           const long long* __restrict__ boff,
                                                           double* __restrict__ bank) {
    const long long i = (long long)blockIdx.x * BANK_BLOCK + threadIdx.x;
    const int v = i < n ? fis_n[i] : 0;
    long long tot;
    const long long off = boff[blockIdx.x] + block_exclusive_scan(v, &tot);
    for (int j = 0; j < v; ++j) {
        bank[3 * (off + j)] = fis_pos[3 * i];
        bank[3 * (off + j) + 1] = fis_pos[3 * i + 1];
        bank[3 * (off + j) + 2] = fis_pos[3 * i + 2];
    }
}

// Births from a bank of *bank_size sites: particle i (id first_id + i) takes
// site floor(xi * B) (xi: first value of counter (pid, 0, TAG_BANK, 0); B - 1
// at xi = 1), the direction and tau of the source-box births.
__global__ void __launch_bounds__(128) k_source_bank(const DevGeom g, long long n, uint64_t first_id, uint32_t seed_lo,
                                                     const double* __restrict__ bank,
                                                     const long long* __restrict__ bank_size, double* __restrict__ buf) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const uint32_t gid = uint32_t(g.gid);
    const long long B = *bank_size;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t pid = uint32_t(first_id + uint64_t(i));
        double x = 0, y = 0, z = 0, u = 0, v = 0, w = 1, tau = 0;
        int st = TRK_E_SOURCE;
        if (B > 0) {
            double xb, unused;
            uniform2(pid, 0, TAG_BANK, 0, seed_lo, gid, xb, unused);
            long long j = (long long)floor(xb * double(B));
            if (j >= B) j = B - 1;
            x = bank[3 * j]; y = bank[3 * j + 1]; z = bank[3 * j + 2];
            if (isotropic(pid, 0, seed_lo, gid, u, v, w)) {
                double unused2, xt;
                uniform2(pid, 0, TAG_SCALARS, 0, seed_lo, gid, unused2, xt);
                tau = -own_log(xt);
                st = 0;
            }
        }
        buf[i] = x; buf[n + i] = y; buf[2 * n + i] = z;
        buf[3 * n + i] = u; buf[4 * n + i] = v; buf[5 * n + i] = w;
        buf[6 * n + i] = tau;
        reinterpret_cast<int*>(buf + 7 * n)[i] = st;
    }
}

__global__ void k_set_double(double* p, double v) { *p = v; }

// A kernel-level status of an inactive cycle (whose counters are scratch)
// is carried to the caller's counters.
__global__ void k_carry_status(const unsigned long long* from, unsigned long long* to) {
    if (from[TRK_K_STATUS] != 0ULL) atomicCAS(to + TRK_K_STATUS, 0ULL, from[TRK_K_STATUS]);
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct PowerLayout {
    size_t parts, fis_pos, fis_n, bsum, bank, tally, cnt, scal, ev, total;
};

PowerLayout power_layout(trk_geom_t g, long long n, const trk_run_opts& o) {
    PowerLayout L;
    const long long nb = (n + BANK_BLOCK - 1) / BANK_BLOCK;
    size_t off = 0;
    L.parts = off; off += al256(particle_bytes(n));
    L.fis_pos = off; off += al256(size_t(n) * 3 * sizeof(double));
    L.fis_n = off; off += al256(size_t(n) * sizeof(int));
    L.bsum = off; off += al256(size_t(nb > 0 ? nb : 1) * sizeof(long long));
    L.bank = off; off += al256(size_t(n) * FISSION_MAX * 3 * sizeof(double));
    L.tally = off; off += al256(size_t(g->n_inst) * sizeof(unsigned long long));
    L.cnt = off; off += al256(TRK_NCOUNTERS * sizeof(unsigned long long));
    L.scal = off; off += 256;   // knorm, nu sum, bank size
    L.ev = off;
    if (o.mode == TRK_MODE_EVENT) {
        const int slots = event_slots(o);
        off += al256(event_work_bytes(slots, o.grid > 0 ? o.grid : event_grid(slots)));
    }
    L.total = off;
    return L;
}

}  // namespace

extern "C" {

trk_status power_iteration_work_bytes(trk_geom_t g, int64_t n, const trk_run_opts* opts, size_t* bytes) {
    if (!valid(g) || n <= 0 || !bytes) return trk_status(set_error(TRK_E_INVALID, "power_iteration_work_bytes: bad arguments"));
    trk_run_opts o;
    trk_default_opts(&o);
    if (opts) o = *opts;
    if (o.mode == TRK_MODE_EVENT) {
        const int slots = event_slots(o);
        if (slots < 32 || slots > 512) return trk_status(set_error(TRK_E_INVALID, "queue_depth must be in [32, 512]"));
    }
    *bytes = power_layout(g, n, o).total;
    return TRK_OK;
}

trk_status power_iteration(trk_geom_t g, int64_t n, int inactive, int cycles, double* dev_k, int64_t* dev_bank,
                           uint64_t* dev_tally, uint64_t* dev_counters, void* dev_work, size_t work_bytes,
                           const trk_run_opts* opts, void* stream) {
    if (!valid(g) || n <= 0 || cycles <= 0 || inactive < 0 || inactive > cycles || !dev_k || !dev_bank || !dev_tally ||
        !dev_counters)
        return trk_status(set_error(TRK_E_INVALID, "power_iteration: bad arguments"));
    if (n > (int64_t(1) << 31) || (long long)cycles * n > (int64_t(1) << 32))
        return trk_status(set_error(TRK_E_INVALID, "power_iteration: cycles * n exceeds 2^32 particle ids"));
    trk_run_opts o;
    trk_default_opts(&o);
    if (opts) o = *opts;
    trk_status st;
    const int tracker = resolve_tracker(g, o.tracker, &st, false, o.mode == TRK_MODE_EVENT);
    if (tracker < 0) return st;
    if (o.precision != TRK_FP64) return trk_status(set_error(TRK_E_UNSUPPORTED, "power_iteration: FP64 only"));
    if (o.mode != TRK_MODE_HISTORY && o.mode != TRK_MODE_EVENT)
        return trk_status(set_error(TRK_E_INVALID, "power_iteration: unknown mode %d", o.mode));
    if (o.max_path > 0.0 && o.max_path < DINF)
        return trk_status(set_error(TRK_E_UNSUPPORTED, "power_iteration: no path cutoff"));
    if (o.mesh_tally && !g->dg.m_n[0])
        return trk_status(set_error(TRK_E_INVALID, "power_iteration: mesh tally given but the geometry has no mesh"));
    if (!(o.p_absorb >= 0.0 && o.p_absorb <= 1.0)) return trk_status(set_error(TRK_E_INVALID, "power_iteration: p_absorb outside [0,1]"));
    if (o.mode == TRK_MODE_EVENT && o.max_rounds < 0) return trk_status(set_error(TRK_E_INVALID, "max_rounds must be >= 0"));
    const PowerLayout L = power_layout(g, n, o);
    if (!dev_work || work_bytes < L.total)
        return trk_status(set_error(TRK_E_NOMEM, "power_iteration: work buffer needs %zu bytes", L.total));
    if ((reinterpret_cast<uintptr_t>(dev_work) & 255) != 0)
        return trk_status(set_error(TRK_E_INVALID, "power_iteration: work buffer must be 256-byte aligned"));
    unsigned char* w = static_cast<unsigned char*>(dev_work);
    double* parts = reinterpret_cast<double*>(w + L.parts);
    double* fis_pos = reinterpret_cast<double*>(w + L.fis_pos);
    int* fis_n = reinterpret_cast<int*>(w + L.fis_n);
    long long* bsum = reinterpret_cast<long long*>(w + L.bsum);
    double* bank = reinterpret_cast<double*>(w + L.bank);
    auto* scratch_tally = reinterpret_cast<unsigned long long*>(w + L.tally);
    auto* scratch_cnt = reinterpret_cast<unsigned long long*>(w + L.cnt);
    double* knorm = reinterpret_cast<double*>(w + L.scal);
    auto* nu_sum = reinterpret_cast<unsigned long long*>(w + L.scal + 8);
    long long* bank_size = reinterpret_cast<long long*>(w + L.scal + 16);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nb = (n + BANK_BLOCK - 1) / BANK_BLOCK;
    const bool csg = tracker == TRK_TRACKER_CSG;
    k_set_double<<<1, 1, 0, s>>>(knorm, 1.0);
    const ParticlesView P = view_of(parts, n);
    for (int c = 0; c < cycles; ++c) {
        const bool active = c >= inactive;
        const uint64_t first = o.first_id + uint64_t(c) * uint64_t(n);
        if (c == 0) {
            k_source<<<persistent_grid(k_source, 128, n, 0), 128, 0, s>>>(g->dg, n, first, uint32_t(o.seed), parts);
        } else {
            k_source_bank<<<persistent_grid(k_source_bank, 128, n, 0), 128, 0, s>>>(g->dg, n, first, uint32_t(o.seed),
                                                                                     bank, bank_size, parts);
        }
        if ((st = launch_error("power_iteration source")) != TRK_OK) return st;
        cudaMemsetAsync(nu_sum, 0, sizeof(unsigned long long), s);
        // an inactive cycle's counters are scratch; its status must start at 0
        if (!active) cudaMemsetAsync(scratch_cnt, 0, TRK_NCOUNTERS * sizeof(unsigned long long), s);
        RunP rp;
        rp.first_id = first;
        rp.max_segments = o.max_segments ? o.max_segments : 1000000ULL;
        rp.p_absorb = o.p_absorb;
        rp.max_path = DINF;
        rp.seed_lo = uint32_t(o.seed);
        rp.trace_cap = 0;
        rp.mesh = active ? reinterpret_cast<unsigned long long*>(o.mesh_tally) : nullptr;
        rp.knorm = knorm;
        rp.fis_pos = fis_pos;
        rp.fis_n = fis_n;
        rp.nu_sum = nu_sum;
        auto* T = active ? reinterpret_cast<unsigned long long*>(dev_tally) : scratch_tally;
        auto* C = active ? reinterpret_cast<unsigned long long*>(dev_counters) : scratch_cnt;
        const int flags = F_FISS | (rp.mesh ? F_MESH : 0);
        if (o.mode == TRK_MODE_EVENT) {
            const int slots = event_slots(o);
            const int grid = o.grid > 0 ? o.grid : event_grid(slots);
            st = launch_event(g, P, n, rp, csg, false, flags, T, C, nullptr, w + L.ev, L.total - L.ev, slots, grid,
                              o.max_rounds, o.sort_interval, s);
        } else {
            const int block = o.block > 0 ? o.block : 128;
            if (block > 128 || (block & 31)) return trk_status(set_error(TRK_E_INVALID, "power_iteration: block must be a multiple of 32, <= 128"));
            if (csg) st = flags & F_MESH ? launch_history<true, false, F_FISS | F_MESH>(g, P, n, rp, T, C, nullptr, nullptr, nullptr, block, o.grid, s)
                                        : launch_history<true, false, F_FISS>(g, P, n, rp, T, C, nullptr, nullptr, nullptr, block, o.grid, s);
            else st = flags & F_MESH ? launch_history<false, false, F_FISS | F_MESH>(g, P, n, rp, T, C, nullptr, nullptr, nullptr, block, o.grid, s)
                                    : launch_history<false, false, F_FISS>(g, P, n, rp, T, C, nullptr, nullptr, nullptr, block, o.grid, s);
        }
        if (st != TRK_OK) return st;
        if (!active) k_carry_status<<<1, 1, 0, s>>>(scratch_cnt, reinterpret_cast<unsigned long long*>(dev_counters));
        k_bank_count<<<unsigned(nb), BANK_BLOCK, 0, s>>>(fis_n, n, bsum);
        k_bank_scan<<<1, BANK_BLOCK, 0, s>>>(bsum, nb, n, nu_sum, knorm, dev_k + c, reinterpret_cast<long long*>(dev_bank) + c,
                                             bank_size, reinterpret_cast<unsigned long long*>(dev_counters));
        k_bank_write<<<unsigned(nb), BANK_BLOCK, 0, s>>>(fis_n, fis_pos, n, bsum, bank);
        if ((st = launch_error("power_iteration bank")) != TRK_OK) return st;
    }
    return TRK_OK;
}

}  // extern "C"
