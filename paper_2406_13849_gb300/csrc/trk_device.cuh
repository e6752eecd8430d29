// trk_device.cuh - device side of the nested-geometry trackers (sm_103a).
//
// Paper: arXiv 2406.13849, Table 1 (find_cell, distance_to_surface,
// move_within_cell, cross_surface, change_direction), Alg. 2-10, Sec. 4.3.
//
// GB300 notes.  The FP64 pipe issues one warp instruction per ~16 SM cycles,
// whatever the active mask; it is the scarce unit.  So:
//  - every FP64 comparison is done as an integer comparison of order keys
//    (okey: the IEEE bit pattern made monotone, -0 equal to +0), exact for
//    non-NaN values, on the integer pipe;
//  - axis-plane senses compare the point's key against the plane's stored
//    key: no FP64 instruction at all;
//  - BVH boxes are FP32, and the point's FP32 bounds (round down / up) are
//    produced from its bits with integer operations;
//  - only the arithmetic of the method's formulas runs on the FP64 pipe, in
//    the order they are written (bit-exact with the FP64 oracle in the
//    --fmad=false build).
#pragma once
#include <cstdint>

#include "trk.h"
#include "trk_internal.h"

namespace trk {
namespace dev {

constexpr double DINF = __builtin_huge_val();
constexpr int MAXMAT = 8;

// ---------------------------------------------------------------------------
// Exact comparisons on the integer pipe
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long okey(double x) { return okey_bits(dbits(x)); }
__device__ __forceinline__ bool d_lt(double a, double b) { return okey(a) < okey(b); }
__device__ __forceinline__ bool d_gt0(double x) { return dbits(x) > 0; }
__device__ __forceinline__ bool d_lt0(double x) { const long long b = dbits(x); return b < 0 && b != (long long)0x8000000000000000ULL; }
__device__ __forceinline__ bool d_ge0(double x) { return !d_lt0(x); }
__device__ __forceinline__ bool d_le0(double x) { return !d_gt0(x); }
__device__ __forceinline__ bool d_eq0(double x) { return (dbits(x) & 0x7fffffffffffffffLL) == 0; }
__device__ __forceinline__ bool d_finite_lt_inf(double x) { return okey(x) < 0x7ff0000000000000LL; }

// FP32 bounds lo <= x <= hi from the bits of x (integer operations only).
__device__ __forceinline__ void f32_bounds(double x, float& lo, float& hi) {
    const unsigned long long b = (unsigned long long)dbits(x);
    const unsigned sign = unsigned(b >> 63);
    const int e = int((b >> 52) & 0x7ff) - 1023 + 127;
    if (e >= 255) {
        lo = sign ? -__int_as_float(0x7f800000) : __int_as_float(0x7f7fffff);
        hi = sign ? -__int_as_float(0x7f7fffff) : __int_as_float(0x7f800000);
        return;
    }
    if (e <= 0) {
        lo = -__int_as_float(0x00800000);
        hi = __int_as_float(0x00800000);
        return;
    }
    const unsigned t = (sign << 31) | (unsigned(e) << 23) | unsigned((b >> 29) & 0x7fffff);
    const unsigned away = t + ((b & 0x1fffffffULL) ? 1u : 0u);
    if (sign) { lo = __uint_as_float(away); hi = __uint_as_float(t); }
    else { lo = __uint_as_float(t); hi = __uint_as_float(away); }
}

// ---------------------------------------------------------------------------
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), counter
// (particle id, event, tag, k), key (seed_lo32, geometry id); two doubles in
// (0, 1] per call: ((u64 >> 11) + 1) * 2^-53.
// ---------------------------------------------------------------------------
enum { TAG_POSITION = 0, TAG_DIRECTION = 1, TAG_SCALARS = 2, TAG_FISSION = 3, TAG_BANK = 4 };

__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += W0; k.y += W1; }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ void uniform2(uint32_t pid, uint32_t event, uint32_t tag, uint32_t k, uint32_t seed_lo,
                                         uint32_t gid, double& a, double& b) {
    const uint4 o = philox10(make_uint4(pid, event, tag, k), make_uint2(seed_lo, gid));
    const uint64_t ua = (uint64_t(o.y) << 32) | o.x;
    const uint64_t ub = (uint64_t(o.w) << 32) | o.z;
    a = double((ua >> 11) + 1) * 0x1.0p-53;
    b = double((ub >> 11) + 1) * 0x1.0p-53;
}

// log x from + - * / only: x = 2^k m, m in [sqrt(1/2), sqrt 2), s = (m-1)/(m+1),
// log m = 2 s (1 + z/3 + z^2/5 + ... + z^13/27), z = s^2 (Horner, highest
// first); log x = k LN2_HI + (log m + k LN2_LO), LN2_HI = ln 2 to 33 bits.
__device__ __forceinline__ double own_log(double x) {
    const uint64_t bits = uint64_t(dbits(x));
    int k = int((bits >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL));
    if (dbits(m) > dbits(1.4142135623730951)) { m = m * 0.5; k += 1; }
    const double s = (m - 1.0) / (m + 1.0);
    const double z = s * s;
    double p = 0x1.2f684bda12f68p-5;                 // 1/27
    p = p * z + 0x1.47ae147ae147bp-5;                // 1/25
    p = p * z + 0x1.642c8590b2164p-5;                // 1/23
    p = p * z + 0x1.8618618618618p-5;                // 1/21
    p = p * z + 0x1.af286bca1af28p-5;                // 1/19
    p = p * z + 0x1.e1e1e1e1e1e1ep-5;                // 1/17
    p = p * z + 0x1.1111111111111p-4;                // 1/15
    p = p * z + 0x1.3b13b13b13b14p-4;                // 1/13
    p = p * z + 0x1.745d1745d1746p-4;                // 1/11
    p = p * z + 0x1.c71c71c71c71cp-4;                // 1/9
    p = p * z + 0x1.2492492492492p-3;                // 1/7
    p = p * z + 0x1.999999999999ap-3;                // 1/5
    p = p * z + 0x1.5555555555555p-2;                // 1/3
    p = p * z + 1.0;
    const double logm = (s + s) * p;
    const double kd = double(k);
    return kd * 0x1.62e42fefp-1 + (logm + kd * 0x1.473de6af278edp-34);
}

// Marsaglia (1972): u, v in (-1, 1], accept 0 < s = u^2+v^2 < 1,
// Omega = (u f, v f, 1 - 2 s), f = 2 sqrt(1 - s); attempt k uses counter
// (pid, event, TAG_DIRECTION, k), at most 64 attempts.
__device__ __forceinline__ bool isotropic(uint32_t pid, uint32_t event, uint32_t seed_lo, uint32_t gid, double& ou,
                                          double& ov, double& ow) {
    for (uint32_t k = 0; k < 64; ++k) {
        double xa, xb;
        uniform2(pid, event, TAG_DIRECTION, k, seed_lo, gid, xa, xb);
        const double u = 2.0 * xa - 1.0;
        const double v = 2.0 * xb - 1.0;
        const double s = u * u + v * v;
        if (d_gt0(s) && dbits(s) < dbits(1.0)) {
            const double f = 2.0 * sqrt(1.0 - s);
            ou = u * f;
            ov = v * f;
            ow = 1.0 - 2.0 * s;
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ uint64_t fnv(uint64_t h, uint64_t w) { return (h ^ w) * 0x100000001b3ULL; }
constexpr uint64_t FNV0 = 0xcbf29ce484222325ULL;

// ---------------------------------------------------------------------------
// Geometry access
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_coef(const DevGeom& g, int s, double& c0, double& c1, double& c2, double& c3) {
    const double2* p = reinterpret_cast<const double2*>(g.s_coef + 4 * s);
    const double2 a = __ldg(p), b = __ldg(p + 1);
    c0 = a.x; c1 = a.y; c2 = b.x; c3 = b.y;
}

// Point with precomputed order keys of its coordinates.
struct Pt {
    double x, y, z;
    long long kx, ky, kz;
};
__device__ __forceinline__ Pt make_pt(double x, double y, double z) {
    Pt p;
    p.x = x; p.y = y; p.z = z;
    p.kx = okey(x); p.ky = okey(y); p.kz = okey(z);
    return p;
}

// Cylinder senses certified in FP32 before any FP64 evaluation (build knob;
// results are unchanged either way).
#ifndef TRK_CYL_SENSE_F32
#define TRK_CYL_SENSE_F32 1
#endif
// and the distance scan's cylinder screen certified in FP32 first
#ifndef TRK_CYL_SCREEN_F32
#define TRK_CYL_SCREEN_F32 1
#endif

// x truncated toward zero to FP32 by integer operations on its bits (no
// FP64 instruction): relative error below 2^-23; |x| < 2^-126 gives 0 and
// |x| >= 2^128 gives NaN (which fails every comparison).
__device__ __forceinline__ float trunc_to_f32(double x) {
    const long long b = __double_as_longlong(x);
    const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
    const int e = int((hi >> 20) & 0x7ffu);
    const unsigned sign = hi & 0x80000000u;
    if (e < 897) return __uint_as_float(sign);
    if (e > 1150) return __uint_as_float(0x7fc00000u);
    return __uint_as_float(sign | (unsigned(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// Sign of a cylinder's f = (qx qx + qy qy) - r r certified in FP32, without
// the FP64 pipe: +1 or -1 when the FP32 value clears the error bound, 0 when
// the FP64 evaluation must decide.  With X = |x| + |x0|, Y = |y| + |y0|: the
// truncations and roundings give |q_f - q| <= 2^-22 X (resp. Y), so
// |f32 - f| <= 2^-20 (X^2 + Y^2 + r^2) with the three FP32 roundings (or
// fewer, contracted), and the FP64 value is within 2^-50 (X^2 + Y^2 + r^2)
// of f; X^2 + Y^2 + r^2 <= 2.01 S for S = x_f^2 + y_f^2 + x0_f^2 + y0_f^2 +
// r^2_f.  |f32| > 2^-15 S (4x the needed 2^-17 S) therefore fixes the sign
// the FP64 evaluation would compute.
__device__ __forceinline__ int cyl_sense_f32(const DevGeom& g, int s, const Pt& p) {
    const float4 cf = __ldg(g.s_coeff + s);   // x0, y0, r*r, r
    const float xf = trunc_to_f32(p.x), yf = trunc_to_f32(p.y);
    const float qx = xf - cf.x, qy = yf - cf.y;
    const float f = (qx * qx + qy * qy) - cf.z;
    const float sm = ((xf * xf + yf * yf) + (cf.x * cf.x + cf.y * cf.y)) + cf.z;
    const float bound = sm * 0x1p-15f;
    return f > bound ? 1 : (f < -bound ? -1 : 0);
}

// FP32 certificate for the distance scan's cylinder screen: true only when
// the FP64 screen (-f > 2 r bd + (2 r bd + r^2) 2^-40) would hold, so the
// candidate is skipped with the same result.  -f64 >= -f32 - 2^-15 S (the
// bound of cyl_sense_f32), and the FP64 right-hand side is at most
// 2 r bd (1 + 2^-19) + (2 r bd + r^2) 2^-38 with r and bd taken from FP32
// copies within 2^-22 of them (a bd beyond FP32 range or a NaN fails).
__device__ __forceinline__ bool cyl_beyond_f32(const DevGeom& g, int s, double x, double y, double bd) {
    const float4 cf = __ldg(g.s_coeff + s);   // x0, y0, r*r, r
    const float xf = trunc_to_f32(x), yf = trunc_to_f32(y), bf = trunc_to_f32(bd);
    const float qx = xf - cf.x, qy = yf - cf.y;
    const float f = (qx * qx + qy * qy) - cf.z;
    const float sm = ((xf * xf + yf * yf) + (cf.x * cf.x + cf.y * cf.y)) + cf.z;
    const float tb = (cf.w + cf.w) * bf;
    const float rhs = tb * (1.0f + 0x1p-19f) + (tb + cf.z) * 0x1p-38f;
    return -f - sm * 0x1p-15f > rhs;
}

// Sense of the point relative to surface s (entry type `type`): f >= 0 is "+".
//   px: x - g >= 0 <=> x >= g (integer key compare);
//   p: ((nx x + ny y) + nz z) - d;  cz: (qx qx + qy qy) - r r, decided in
//   FP32 when the FP32 value certifies the sign (cyl_sense_f32).
__device__ __forceinline__ int sense_at(const DevGeom& g, int s, int type, const Pt& p) {
    if (type <= S_PZ) {
        const long long kg = __ldg(g.s_key + s);
        const long long kp = type == S_PX ? p.kx : (type == S_PY ? p.ky : p.kz);
        return kp >= kg ? 1 : -1;
    }
#if TRK_CYL_SENSE_F32
    if (type == S_CZ) {
        const int sf = cyl_sense_f32(g, s, p);
        if (sf != 0) return sf;
    }
#endif
    double c0, c1, c2, c3;
    load_coef(g, s, c0, c1, c2, c3);
    double f;
    if (type == S_P) {
        f = ((c0 * p.x + c1 * p.y) + c2 * p.z) - c3;
    } else {
        const double qx = p.x - c0, qy = p.y - c1;
        f = (qx * qx + qy * qy) - c3;
    }
    return d_ge0(f) ? 1 : -1;
}

// Distance to surface s, leaving its `side` (+1/-1) of it; `on` is the logical
// on-surface state.  Negative results (a point a rounding error outside the
// cell) become 0; INF means no hit.
//  planes: only the face the direction leaves through is a candidate;
//    px: t = (g - x) * inv_u; p: t = (d - ((nx x + ny y) + nz z)) /
//    ((nx u + ny v) + nz w); a plane the particle is on is never hit again.
//  cz: a = u u + v v, b = qx u + qy v; on it and logically inside:
//    t = -2 b / a if b < 0, else no hit; on it and outside: no hit;
//    otherwise c = f, disc = b b - a c, no hit if a == 0 or disc <= 0;
//    inside: t = b <= 0 ? (-b + sqrt disc) / a : -c / (b + sqrt disc);
//    outside: hit only if b < 0, t = c / (-b + sqrt disc).
struct Dir {
    double u, v, w, iu, iv, iw;
};

__device__ __forceinline__ double surface_distance(const DevGeom& g, int s, int type, int side, bool on,
                                                   double x, double y, double z, const Dir& d) {
    double t;
    if (type <= S_PZ) {
        if (on) return DINF;
        const double dd = type == S_PX ? d.u : (type == S_PY ? d.v : d.w);
        const bool leaves = side > 0 ? d_lt0(dd) : d_gt0(dd);
        if (!leaves) return DINF;
        const double gval = __ldg(g.s_coef + 4 * s);
        const double xx = type == S_PX ? x : (type == S_PY ? y : z);
        const double ii = type == S_PX ? d.iu : (type == S_PY ? d.iv : d.iw);
        t = (gval - xx) * ii;
    } else if (type == S_P) {
        if (on) return DINF;
        double c0, c1, c2, c3;
        load_coef(g, s, c0, c1, c2, c3);
        const double den = (c0 * d.u + c1 * d.v) + c2 * d.w;
        const bool leaves = side > 0 ? d_lt0(den) : d_gt0(den);
        if (!leaves) return DINF;
        const double num = c3 - ((c0 * x + c1 * y) + c2 * z);
        t = num / den;
    } else {
        double c0, c1, c2, c3;
        load_coef(g, s, c0, c1, c2, c3);
        const double qx = x - c0, qy = y - c1;
        const double a = d.u * d.u + d.v * d.v;
        const double b = qx * d.u + qy * d.v;
        // every case is one quotient num / den, so lanes that take different
        // cases still share one square root and one division
        double num, den;
        if (on) {
            if (side < 0 && d_lt0(b)) { num = -2.0 * b; den = a; }
            else return DINF;
        } else {
            const double c = (qx * qx + qy * qy) - c3;
            if (d_eq0(a)) return DINF;
            const double disc = b * b - a * c;
            if (d_le0(disc)) return DINF;
            if (side > 0 && !d_lt0(b)) return DINF;
            const double sq = sqrt(disc);
            if (side < 0) {
                if (d_le0(b)) { num = -b + sq; den = a; }
                else { num = -c; den = b + sq; }
            } else {
                num = c; den = -b + sq;
            }
        }
        t = num / den;
    }
    if (d_lt0(t)) t = 0.0;
    return t;
}

// Cell test: all senses hold; the crossed surface xs (if >= 0) is taken
// logically with sense xsn instead of being evaluated.
// The plane-pair part of the cell test, out of line: only cells with
// general planes (hex elements) call it, and the kernels of geometries
// without them keep a smaller instruction footprint.
static __device__ __noinline__ bool pairs_hold(const DevGeom& g, int c, const Pt& p, int xs, int xsn) {
    const int4 p0 = __ldg(g.c_pair + 2 * c), p1 = __ldg(g.c_pair + 2 * c + 1);
    const int pe[6] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (pe[k] < 0) continue;
        const int e = __ldg(g.cs + pe[k]);
        const int sf = cs_surface(e), sn = cs_side(e);
        if (sf == xs) {
            if (sn != xsn) return false;
        } else if (sense_at(g, sf, S_P, p) != sn) {
            return false;
        }
    }
    return true;
}

#ifndef TRK_HOLDS_INLINE
#define TRK_HOLDS_INLINE __forceinline__
#endif
static __device__ TRK_HOLDS_INLINE bool cell_holds(const DevGeom& g, int c, const Pt& p, int xs, int xsn) {
    const int2 rg = __ldg(g.c_range + c);
    if (rg.y & CS_SLAB_FLAG) {
        // slab view: per dimension x >= g_lo ("+" side of the lower face) and
        // x < g_hi ("-" side of the upper face), as order-key compares, then
        // the remaining entries; the same conjunction as the entry loop below
        const longlong2* K = g.c_slabk + 3 * c;
        const longlong2 kx = __ldg(K), ky = __ldg(K + 1), kz = __ldg(K + 2);
        const int4 s0 = __ldg(g.c_slabs + 2 * c), s1 = __ldg(g.c_slabs + 2 * c + 1);
        const long long lo3[3] = {kx.x, ky.x, kz.x}, hi3[3] = {kx.y, ky.y, kz.y};
        const int ls3[3] = {s0.x, s0.z, s1.x}, hs3[3] = {s0.y, s0.w, s1.y};
        const long long kp3[3] = {p.kx, p.ky, p.kz};
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const bool lo_ok = (ls3[d] >= 0 && ls3[d] == xs) ? (xsn > 0) : (kp3[d] >= lo3[d]);
            const bool hi_ok = (hs3[d] >= 0 && hs3[d] == xs) ? (xsn < 0) : (kp3[d] < hi3[d]);
            ok = ok && lo_ok && hi_ok;
        }
        if (!ok) return false;
        if ((rg.y & CS_PAIR_FLAG) && !pairs_hold(g, c, p, xs, xsn)) return false;
        const int2 rr = __ldg(g.c_rest + c);
        for (int k = 0; k < rr.y; ++k) {
            const int e = __ldg(g.cs + __ldg(g.rest_e + rr.x + k));
            const int sf = cs_surface(e), sn = cs_side(e);
            if (sf == xs) {
                if (sn != xsn) return false;
            } else if (sense_at(g, sf, cs_type(e), p) != sn) {
                return false;
            }
        }
        return true;
    }
    const int cnt = rg.y & CS_COUNT_MASK;
    for (int k = 0; k < cnt; ++k) {
        const int e = __ldg(g.cs + rg.x + k);
        const int s = cs_surface(e), sn = cs_side(e);
        if (s == xs) {
            if (sn != xsn) return false;
        } else if (sense_at(g, s, cs_type(e), p) != sn) {
            return false;
        }
    }
    return true;
}

// Walk of universe u's BVH (Sec. 4.3) for the first cell holding the point,
// excluding cell `ex`: each node load tests both children's boxes, the walk
// descends left before right (the right child waits on a short stack when
// the point is in both boxes) and stops at the first holding cell, which is
// the preorder walk's result.  Kept out of line (TRK_OUTLINE_SEARCH): one copy
// instead of one per call site keeps the event kernel's instruction
// footprint small, which measured 36% faster for the CSG tracker.
#ifndef TRK_OUTLINE_SEARCH
#define TRK_OUTLINE_SEARCH 1
#endif
#if TRK_OUTLINE_SEARCH
#define TRK_SEARCH_INLINE __noinline__
#else
#define TRK_SEARCH_INLINE __forceinline__
#endif
// Kernels that stage the BVH nodes in shared memory (TRK_BVH_SMEM, the
// event kernels) leave their address here at launch, or nullptr when the
// geometry's nodes do not fit; the walk then reads the staged copy.
#ifndef TRK_BVH_SMEM
#define TRK_BVH_SMEM 0
#endif
#if TRK_BVH_SMEM
__shared__ const BvhNode* s_bvh_nodes;
#endif

// One walk for both copies: in the event kernels `nodes` is a generic
// pointer to either the shared-memory copy or the global array (plain loads
// serve both), elsewhere the global array read through the read-only path.
__device__ __forceinline__ int bvh_walk(const DevGeom& g, const BvhNode* nodes, int root, const Pt& p, int ex, int xs,
                                        int xsn) {
    float xl, xh, yl, yh, zl, zh;
    f32_bounds(p.x, xl, xh);
    f32_bounds(p.y, yl, yh);
    f32_bounds(p.z, zl, zh);
    int stack[BVH_STACK];
    int sp = 0;
    int ref = root;
    for (;;) {
        if (ref >= 0) {
            const float4* np = reinterpret_cast<const float4*>(nodes + ref);
#if TRK_BVH_SMEM
            const float4 a = np[0], b = np[1], c = np[2];
            const int4 r = *reinterpret_cast<const int4*>(np + 3);
#else
            const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
            const int4 r = __ldg(reinterpret_cast<const int4*>(np + 3));
#endif
            // child 0: lo (a.x, a.y, a.z), hi (a.w, b.x, b.y); child 1: lo (b.z, b.w, c.x), hi (c.y, c.z, c.w)
            const bool in0 = xh >= a.x && xl <= a.w && yh >= a.y && yl <= b.x && zh >= a.z && zl <= b.y;
            const bool in1 = xh >= b.z && xl <= c.y && yh >= b.w && yl <= c.z && zh >= c.x && zl <= c.w;
            if (in0) {
                if (in1 && sp < BVH_STACK) stack[sp++] = r.y;
                ref = r.x;
                continue;
            }
            if (in1) {
                ref = r.y;
                continue;
            }
        } else {
            const int leaf = -1 - ref;
            const int first = leaf >> 4, cnt = leaf & 15;
            for (int k = 0; k < cnt; ++k) {
                const int c = __ldg(g.leaf_cells + first + k);
                if (c != ex && cell_holds(g, c, p, xs, xsn)) return c;
            }
        }
        if (sp == 0) return -1;
        ref = stack[--sp];
    }
}

static __device__ TRK_SEARCH_INLINE int bvh_search(const DevGeom& g, int root, const Pt& p, int ex, int xs, int xsn) {
#if TRK_BVH_SMEM
    return bvh_walk(g, s_bvh_nodes ? s_bvh_nodes : g.nodes, root, p, ex, xs, xsn);
#else
    return bvh_walk(g, g.nodes, root, p, ex, xs, xsn);
#endif
}

// Walk of universe u's bounding interval hierarchy (Sec. 4.3): at each node
// both edge conditions are tested (the half-spaces may overlap): left if the
// point can be at or below clip_l along the node's axis, right if it can be
// at or above clip_r; left before right, first holding cell returned.
static __device__ TRK_SEARCH_INLINE int bih_search(const DevGeom& g, int root, const Pt& p, int ex, int xs, int xsn) {
    float lo3[3], hi3[3];
    f32_bounds(p.x, lo3[0], hi3[0]);
    f32_bounds(p.y, lo3[1], hi3[1]);
    f32_bounds(p.z, lo3[2], hi3[2]);
    int stack[BVH_STACK];
    int sp = 0;
    int ref = root;
    for (;;) {
        if (ref >= 0) {
            const float4 nd = __ldg(reinterpret_cast<const float4*>(g.bih + ref));
            const int r0 = __float_as_int(nd.z), r1a = __float_as_int(nd.w);
            const int ax = r1a & 3, r1 = r1a >> 2;
            const float pl = ax == 0 ? lo3[0] : (ax == 1 ? lo3[1] : lo3[2]);
            const float ph = ax == 0 ? hi3[0] : (ax == 1 ? hi3[1] : hi3[2]);
            const bool in0 = pl <= nd.x, in1 = ph >= nd.y;
            if (in0) {
                if (in1 && sp < BVH_STACK) stack[sp++] = r1;
                ref = r0;
                continue;
            }
            if (in1) {
                ref = r1;
                continue;
            }
        } else {
            const int leaf = -1 - ref;
            const int first = leaf >> 4, cnt = leaf & 15;
            for (int k = 0; k < cnt; ++k) {
                const int c = __ldg(g.leaf_cells + first + k);
                if (c != ex && cell_holds(g, c, p, xs, xsn)) return c;
            }
        }
        if (sp == 0) return -1;
        ref = stack[--sp];
    }
}

// First cell of universe u (CSG view) holding the point, excluding cell `ex`:
// linear scan for small universes (Alg. 3/4), otherwise the walk of the
// geometry's acceleration structure (BVH, or BIH with "accel": "bih").
__device__ __forceinline__ int csg_search(const DevGeom& g, int u, const Pt& p, int ex, int xs, int xsn) {
    const int4 ui = __ldg(g.u_info + u);
    if (ui.z < 0) {
        for (int c = ui.x; c < ui.x + ui.y; ++c) {
            if (c == ex) continue;
            if (cell_holds(g, c, p, xs, xsn)) return c;
        }
        return -1;
    }
    if (g.accel) return bih_search(g, __ldg(g.u_bih + u), p, ex, xs, xsn);
    return bvh_search(g, ui.z, p, ex, xs, xsn);
}

// Alg. 5: element index in one dimension by binary search on the planes'
// order keys; element i holds g_i <= x < g_{i+1}; a root array has nothing
// outside [g_0, g_n), a non-root array clamps.
__device__ __forceinline__ int rect_index(const long long* gk, int n, long long kx, bool root) {
    if (root && (!(__ldg(gk) <= kx) || !(kx < __ldg(gk + n)))) return -1;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(gk + mid) <= kx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Particle state (registers)
// ---------------------------------------------------------------------------
struct Lv {
    int u, cell, i, j, k, off;
    double tx, ty, tz;
};

struct St {
    double x, y, z, tau;
    Dir d;
    int nlev, on_lev, on_surf, mat;
    Lv lv[MAXL];
};

// Collision distance in the fast build by the reciprocal cross section
// (build knob; the exact build always divides).
#ifndef TRK_FAST_RSIGMA
#define TRK_FAST_RSIGMA 1
#endif

// Inlining of the less frequent steps (build knobs, measured per kernel):
// out of line they leave the hot flight code a smaller footprint, at the
// price of a call.
#ifndef TRK_COLLIDE_INLINE
#define TRK_COLLIDE_INLINE __forceinline__
#endif
#ifndef TRK_FIND_INLINE
#define TRK_FIND_INLINE __forceinline__
#endif
#ifndef TRK_CROSS_INLINE
#define TRK_CROSS_INLINE __forceinline__
#endif

// Level access by a run-time level index.  The level stack stays in
// registers (an indexed array would go to local memory); these select among
// the MAXL entries, so a loop over levels can keep one copy of its body
// instead of MAXL unrolled copies (the kernels' instruction footprint is
// what the instruction caches see).
static_assert(MAXL == 4, "level selects assume four levels");
__device__ __forceinline__ Lv lv_get(const St& s, int l) {
    Lv L = s.lv[0];
    if (l == 1) L = s.lv[1];
    if (l == 2) L = s.lv[2];
    if (l == 3) L = s.lv[3];
    return L;
}
__device__ __forceinline__ void lv_set(St& s, int l, const Lv& L) {
    if (l == 0) s.lv[0] = L;
    if (l == 1) s.lv[1] = L;
    if (l == 2) s.lv[2] = L;
    if (l == 3) s.lv[3] = L;
}
__device__ __forceinline__ void lv_set_u(St& s, int l, int u) {
    if (l == 0) s.lv[0].u = u;
    if (l == 1) s.lv[1].u = u;
    if (l == 2) s.lv[2].u = u;
    if (l == 3) s.lv[3].u = u;
}
__device__ __forceinline__ double sel4(int l, double a0, double a1, double a2, double a3) {
    double v = a0;
    if (l == 1) v = a1;
    if (l == 2) v = a2;
    if (l == 3) v = a3;
    return v;
}

__device__ __forceinline__ void set_inverse(Dir& d) {
    d.iu = 1.0 / d.u;
    d.iv = 1.0 / d.v;
    d.iw = 1.0 / d.w;
}

__device__ __forceinline__ void clear_levels(St& s) {
    s.nlev = 0; s.mat = 0; s.on_lev = -1; s.on_surf = -1;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        s.lv[l].u = 0; s.lv[l].cell = 0; s.lv[l].i = s.lv[l].j = s.lv[l].k = 0; s.lv[l].off = 0;
        s.lv[l].tx = s.lv[l].ty = s.lv[l].tz = 0.0;
    }
}

__device__ __forceinline__ int instance(const St& s) {
    int t = 0;
#pragma unroll
    for (int l = 0; l < MAXL; ++l)
        if (l < s.nlev) t += s.lv[l].off;
    return t;
}

// Local position at level `lev`: global minus translations of levels
// 0..lev-1, component by component in level order.
__device__ __forceinline__ void local_at(const St& s, int lev, double& x, double& y, double& z) {
    x = s.x; y = s.y; z = s.z;
#pragma unroll
    for (int l = 0; l < MAXL - 1; ++l) {
        if (l < lev) { x = x - s.lv[l].tx; y = y - s.lv[l].ty; z = z - s.lv[l].tz; }
    }
}

// Sets level L to rect element (i,j,k) of lattice `lat`; returns the daughter.
__device__ __forceinline__ int enter_element(const DevGeom& g, Lv& L, int lat, int i, int j, int k) {
    const int4 dm = __ldg(g.l_dim + lat), of = __ldg(g.l_off + lat);
    const int e = i + dm.x * (j + dm.y * k);
    L.i = i; L.j = j; L.k = k;
    L.cell = e;
    L.off = __ldg(g.l_eoff + of.w + e);
    L.tx = __ldg(g.l_ctr + of.x + i);
    L.ty = __ldg(g.l_ctr + of.y + j);
    L.tz = __ldg(g.l_ctr + of.z + k);
    return __ldg(g.l_fill + of.w + e);
}

__device__ __forceinline__ int enter_cell(const DevGeom& g, Lv& L, int c) {
    L.cell = c;
    L.off = __ldg(g.c_off + c);
    L.tx = __ldg(g.c_tr + 3 * c);
    L.ty = __ldg(g.c_tr + 3 * c + 1);
    L.tz = __ldg(g.c_tr + 3 * c + 2);
    return __ldg(g.c_fill + c);
}

// Array tracker, hex lattice h of universe u: the element holding the point
// by closed form.  Axial coordinates from the inverse lattice matrix, cube
// rounding to the nearest element, then the exact test of that element's
// pseudo-array cell (its face planes' senses, as the CSG search evaluates
// them) and of its six neighbours; if none holds, the universe search.  In a
// lattice whose cells partition its region the holding cell is unique, so
// this returns what the pseudo-array scan returns.  Out of line: inlined at
// every find site it would put its cell tests into the instruction
// footprint of array-tracker kernels whose geometries have no hex arrays.
static __device__ __noinline__ int hex_find(const DevGeom& g, int h, int u, const Pt& p) {
    const double2* hp = reinterpret_cast<const double2*>(g.hx + h);
    const double2 m0 = __ldg(hp), m1 = __ldg(hp + 1);
    const int4 hi = __ldg(reinterpret_cast<const int4*>(g.hx + h) + 2);
    const int R = hi.x;
    const double qf = m0.x * p.x + m0.y * p.y, rf = m1.x * p.x + m1.y * p.y;
    const double sf = -qf - rf;
    double qr = rint(qf), rr = rint(rf);
    const double sr = rint(sf);
    const double dq = fabs(qr - qf), dr = fabs(rr - rf), ds = fabs(sr - sf);
    if (dq > dr && dq > ds) qr = -rr - sr;
    else if (dr > ds) rr = -qr - sr;
    const int q0 = int(qr), r0 = int(rr);
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        // the candidate, then its neighbours (q+1, q-1, r+1, r-1, (q+1, r-1), (q-1, r+1))
        const int q = q0 + (k == 1 || k == 5 ? 1 : (k == 2 || k == 6 ? -1 : 0));
        const int r = r0 + (k == 3 || k == 6 ? 1 : (k == 4 || k == 5 ? -1 : 0));
        if (max(abs(q), max(abs(r), abs(q + r))) > R) continue;
        const int e = __ldg(g.hx_row + hi.z + r + R) + q - max(-R, -R - r);
        const int c = hi.y + e;
        if (cell_holds(g, c, p, -1, 0)) return c;
    }
    return csg_search(g, u, p, -1, -1, 0);
}

// Tracker kinds of the tracking templates: the array tracker (rect arrays by
// index, hex arrays by hex_find), the CSG tracker (every universe through
// its cells), and the dynamic-polymorphism tracker (rect arrays and CSG
// universes as two tracker objects reached through virtual calls per level,
// the paper's DP method, Sec. 4.1; the per-level work is the array
// tracker's, hex arrays are CSG universes).  A `bool` CSG argument converts
// to the first two.
enum { TK_RECT = 0, TK_CSG = 1, TK_DP = 2 };

// The per-level steps, shared by the templates below and the DP tracker
// objects.  find_cell in one rect array level (Alg. 5): false if the point is
// outside a root array.
__device__ __forceinline__ bool find_level_rect(const DevGeom& g, Lv& L, int lat, const Pt& p, bool root, int& dau) {
    const int4 dm = __ldg(g.l_dim + lat), of = __ldg(g.l_off + lat);
    const int i = rect_index(g.l_gkey + of.x, dm.x, p.kx, root);
    const int j = rect_index(g.l_gkey + of.y, dm.y, p.ky, root);
    const int k = rect_index(g.l_gkey + of.z, dm.z, p.kz, root);
    if (i < 0 || j < 0 || k < 0) return false;
    dau = enter_element(g, L, lat, i, j, k);
    return true;
}

// find_cell in one CSG level (Alg. 3), or a hex array by hex_find when
// `hex` (-2 - lattice index) is given: false if no cell holds the point.
__device__ __forceinline__ bool find_level_csg(const DevGeom& g, Lv& L, int hex, const Pt& p, int& dau) {
    const int c = hex <= -2 ? hex_find(g, -2 - hex, L.u, p) : csg_search(g, L.u, p, -1, -1, 0);
    if (c < 0) return false;
    dau = enter_cell(g, L, c);
    return true;
}

struct Hit;
struct Tracker;
__device__ __forceinline__ const Tracker* get_tracker(const DevGeom& g, const int4& ui);
__device__ __forceinline__ bool dp_find(const Tracker* t, const DevGeom& g, Lv& L, int lat, const Pt& p, bool root,
                                        int& dau);

// Alg. 7 from level `start` downward (rect view for rect arrays unless CSG).
// Returns 0 on success, -1 if no cell holds the point.
template <int TK>
__device__ TRK_FIND_INLINE int find_from(const DevGeom& g, St& s, int start) {
    constexpr bool CSG = TK == TK_CSG;
    if (start < 0 || start >= MAXL) return -1;
    double x, y, z;
    local_at(s, start, x, y, z);
#pragma unroll 1
    for (int l = start; l < MAXL; ++l) {
        Lv L = lv_get(s, l);
        const int4 ui = __ldg(g.u_info + L.u);
        const Pt p = make_pt(x, y, z);
        int dau;
        bool ok;
        if constexpr (TK == TK_DP) ok = dp_find(get_tracker(g, ui), g, L, ui.w, p, l == 0, dau);
        else if (!CSG && ui.w >= 0) ok = find_level_rect(g, L, ui.w, p, l == 0, dau);
        else ok = find_level_csg(g, L, CSG ? -1 : ui.w, p, dau);
        if (!ok) return -1;
        lv_set(s, l, L);
        if (dau < 0) {
            s.nlev = l + 1;
            s.mat = ~dau;
            return 0;
        }
        if (l + 1 >= MAXL) return -1;
        x = x - L.tx; y = y - L.ty; z = z - L.tz;
        lv_set_u(s, l + 1, dau);
    }
    return -1;
}

struct Hit {
    double d;
    int level, surf, side, dim, dsign, entry;
};

// distance_to_surface in one rect array level (Table 1): per dimension the
// face the direction leaves through, outer faces only at the root; candidate
// c with order key ck (kept when smaller).
__device__ __forceinline__ void dist_level_rect(const DevGeom& g, const St& s, int l, const Lv& L, int lat, double x,
                                                double y, double z, Hit& c, long long& ck) {
    const int4 dm = __ldg(g.l_dim + lat), of = __ldg(g.l_off + lat);
    const int n3[3] = {dm.x, dm.y, dm.z};
    const int o3[3] = {of.x, of.y, of.z};
    const int i3[3] = {L.i, L.j, L.k};
    const double p3[3] = {x, y, z};
    const double d3[3] = {s.d.u, s.d.v, s.d.w};
    const double v3[3] = {s.d.iu, s.d.iv, s.d.iw};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double t = DINF;
        int sg = 0;
        if (d_gt0(d3[d])) {
            if (i3[d] < n3[d] - 1 || l == 0) { t = (__ldg(g.l_grid + o3[d] + i3[d] + 1) - p3[d]) * v3[d]; sg = 1; }
        } else if (d_lt0(d3[d])) {
            if (i3[d] > 0 || l == 0) { t = (__ldg(g.l_grid + o3[d] + i3[d]) - p3[d]) * v3[d]; sg = -1; }
        }
        if (sg != 0) {
            if (d_lt0(t)) t = 0.0;
            const long long tk = okey(t);
            if (tk < ck) {
                ck = tk; c.d = t; c.level = l; c.surf = -1 - (2 * d + (sg > 0)); c.dim = d; c.dsign = sg;
                c.side = 0; c.entry = -1;
            }
        }
    }
}

// distance_to_surface in one CSG level (Table 1): the cell's surfaces (slab
// and pair views first where the cell has them); hk, hd: the running best
// of the levels below, for the cylinder screen.
__device__ __forceinline__ void dist_level_csg(const DevGeom& g, const St& s, int l, const Lv& L, double x, double y,
                                               double z, long long hk, double hd, Hit& c, long long& ck) {
    const long long kinf = okey(DINF);
    const int2 rg = __ldg(g.c_range + L.cell);
    int first = rg.x, cnt = rg.y & CS_COUNT_MASK;
    const int* ents = g.cs;
    bool by_index = false;
    if (rg.y & CS_SLAB_FLAG) {
        // Slab view: per dimension the one axis face the direction
        // leaves through, as in the rect tracker; then the cell's other
        // surfaces.  Ties go to the lower entry index, which is the
        // cell-order scan's result.
        const int4 s0 = __ldg(g.c_slab0 + L.cell), s1 = __ldg(g.c_slab1 + L.cell);
        const int lo3[3] = {s0.x, s0.z, s1.x};
        const int hi3[3] = {s0.y, s0.w, s1.y};
        const double p3[3] = {x, y, z};
        const double d3[3] = {s.d.u, s.d.v, s.d.w};
        const double v3[3] = {s.d.iu, s.d.iv, s.d.iw};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int e = d_gt0(d3[d]) ? hi3[d] : (d_lt0(d3[d]) ? lo3[d] : -1);
            if (e < 0) continue;
            const int sid = cs_surface(__ldg(g.cs + e));
            if (s.on_lev == l && s.on_surf == sid) continue;
            double t = (__ldg(g.s_coef + 4 * sid) - p3[d]) * v3[d];
            if (d_lt0(t)) t = 0.0;
            const long long tk = okey(t);
            if (tk < ck || (tk == ck && c.level >= 0 && e < c.entry)) {
                ck = tk; c.d = t; c.level = l; c.surf = sid; c.side = d_gt0(d3[d]) ? -1 : 1;
                c.dim = -1; c.dsign = 0; c.entry = e;
            }
        }
        if (rg.y & CS_PAIR_FLAG) {
            // plane pairs: per pair the one face the direction leaves
            // through (n.u < 0: the "+" entry), the S_P distance of
            // surface_distance
            const int4 p0 = __ldg(g.c_pair + 2 * L.cell), p1 = __ldg(g.c_pair + 2 * L.cell + 1);
            const int lo3p[3] = {p0.x, p0.z, p1.x};
            const int hi3p[3] = {p0.y, p0.w, p1.y};
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const int ea = lo3p[f] >= 0 ? lo3p[f] : hi3p[f];
                if (ea < 0) continue;
                double c0, c1, c2, c3;
                load_coef(g, cs_surface(__ldg(g.cs + ea)), c0, c1, c2, c3);
                const double den = (c0 * s.d.u + c1 * s.d.v) + c2 * s.d.w;
                const int e = d_lt0(den) ? lo3p[f] : (d_gt0(den) ? hi3p[f] : -1);
                if (e < 0) continue;
                const int sid = cs_surface(__ldg(g.cs + e));
                if (s.on_lev == l && s.on_surf == sid) continue;
                const double d3c = __ldg(g.s_coef + 4 * sid + 3);
                double t = (d3c - ((c0 * x + c1 * y) + c2 * z)) / den;
                if (d_lt0(t)) t = 0.0;
                const long long tk = okey(t);
                if (tk < ck || (tk == ck && c.level >= 0 && e < c.entry)) {
                    ck = tk; c.d = t; c.level = l; c.surf = sid; c.side = d_lt0(den) ? 1 : -1;
                    c.dim = -1; c.dsign = 0; c.entry = e;
                }
            }
        }
        const int2 rr = __ldg(g.c_rest + L.cell);
        first = rr.x; cnt = rr.y; ents = g.rest_e; by_index = true;
    }
    // remaining entries (all of them for a cell without a view)
    for (int k = 0; k < cnt; ++k) {
        const int ei = by_index ? __ldg(ents + first + k) : first + k;
        const int e = __ldg(g.cs + ei);
        const int sid = cs_surface(e), side = cs_side(e), type = cs_type(e);
        const bool on = (s.on_lev == l && s.on_surf == sid);
        if (type == S_CZ && side < 0 && !on && (hk != kinf || ck != kinf)) {
            const double bd = ck < hk ? c.d : hd;
#if TRK_CYL_SCREEN_F32
            if (cyl_beyond_f32(g, sid, x, y, bd)) continue;
#endif
            double c0, c1, c2, c3;
            load_coef(g, sid, c0, c1, c2, c3);
            const double qx = x - c0, qy = y - c1;
            const double f = (qx * qx + qy * qy) - c3;
            if (d_lt0(f)) {
                const double tb = (c2 + c2) * bd;
                const double rhs = tb + (tb + c3) * 0x1p-40;
                if (okey(-f) > okey(rhs)) continue;
            }
        }
        const double t = surface_distance(g, sid, type, side, on, x, y, z, s.d);
        const long long tk = okey(t);
        if (tk < ck || (tk == ck && c.level >= 0 && ei < c.entry)) {
            ck = tk; c.d = t; c.level = l; c.surf = sid; c.side = side; c.dim = -1; c.dsign = 0; c.entry = ei;
        }
    }
}

__device__ __forceinline__ void dp_distance(const Tracker* t, const DevGeom& g, const St& s, int l, const Lv& L, int lat,
                                            double x, double y, double z, long long hk, double hd, Hit& c,
                                            long long& ck);

// distance_to_surface over the levels (Table 1, Alg. 2): the smallest
// distance wins; a tie goes to the top-most level, and within a level to the
// first candidate in the level's order (rect levels: x, y, z faces in the
// direction of flight, outer faces only at the root; CSG levels: the cell's
// surfaces in cell order, which for a slab cell means the lower entry index).
// The levels are scanned bottom-up, each level's winner replacing the running
// best on a tie, which gives the same winner as a top-down scan with strict
// '<'.  Scanning bottom-up lets an upper level skip a cylinder it is inside
// of when the cylinder certainly lies beyond the running best: a ray from a
// point at distance rho from the axis of a cylinder of radius r travels at
// least r - rho >= (r^2 - rho^2) / (2 r) before reaching it.  The test keeps
// a relative margin of 2^-40 over the rounding errors of c = rho^2 - r^2 and
// of the distance formula (both a few ulp: inside a cylinder disc >= b^2), so
// a skipped candidate is never the winner and the result is unchanged.
template <int TK>
__device__ __forceinline__ Hit distance_to_boundary(const DevGeom& g, const St& s) {
    constexpr bool CSG = TK == TK_CSG;
    Hit h;
    h.d = DINF; h.level = -1; h.surf = -1; h.side = 0; h.dim = -1; h.dsign = 0; h.entry = -1;
    const long long kinf = okey(DINF);
    long long hk = kinf;
    double lx[MAXL], ly[MAXL], lz[MAXL];
    lx[0] = s.x; ly[0] = s.y; lz[0] = s.z;
#pragma unroll
    for (int l = 1; l < MAXL; ++l) {
        if (l < s.nlev) {
            lx[l] = lx[l - 1] - s.lv[l - 1].tx; ly[l] = ly[l - 1] - s.lv[l - 1].ty; lz[l] = lz[l - 1] - s.lv[l - 1].tz;
        } else {
            lx[l] = lx[l - 1]; ly[l] = ly[l - 1]; lz[l] = lz[l - 1];
        }
    }
    // the loop runs over all MAXL levels so that the lanes of a warp stay
    // on the same level (a lane with fewer levels idles through the deeper
    // ones) instead of each starting at its own deepest level
#pragma unroll 1
    for (int l = MAXL - 1; l >= 0; --l) {
        if (l >= s.nlev) continue;
        const double x = sel4(l, lx[0], lx[1], lx[2], lx[3]);
        const double y = sel4(l, ly[0], ly[1], ly[2], ly[3]);
        const double z = sel4(l, lz[0], lz[1], lz[2], lz[3]);
        const Lv L = lv_get(s, l);
        Hit c;
        c.d = DINF; c.level = -1; c.surf = -1; c.side = 0; c.dim = -1; c.dsign = 0; c.entry = -1;
        long long ck = kinf;
        const int4 ui = __ldg(g.u_info + L.u);
        if constexpr (TK == TK_DP) dp_distance(get_tracker(g, ui), g, s, l, L, ui.w, x, y, z, hk, h.d, c, ck);
        else if (!CSG && ui.w >= 0) dist_level_rect(g, s, l, L, ui.w, x, y, z, c, ck);
        else dist_level_csg(g, s, l, L, x, y, z, hk, h.d, c, ck);
        if (c.level >= 0 && ck <= hk) { hk = ck; h = c; }
    }
    return h;
}

// ---------------------------------------------------------------------------
// FP32-local distances.  Every level's coordinates come from the FP64 chain
// (global position minus the FP64 translations), rounded once to FP32 in the
// frame where they are small: array and slab faces are measured in the
// element's own frame (|coordinates| < half a pitch), other CSG surfaces in
// their universe's frame.  All distance formulas then run in FP32.  The two
// smallest candidates are kept; when they are within CLOSE_REL of each other
// (or of the collision distance) the step is redone exactly in FP64.
// ---------------------------------------------------------------------------
constexpr float CLOSE_REL = 2e-5f;
constexpr float FINF = __builtin_huge_valf();

struct DirF {
    float u, v, w, iu, iv, iw;
};

__device__ __forceinline__ DirF dir_f32(const Dir& d) {
    DirF f;
    f.u = float(d.u); f.v = float(d.v); f.w = float(d.w);
    f.iu = 1.0f / f.u; f.iv = 1.0f / f.v; f.iw = 1.0f / f.w;
    return f;
}

// `ill` is set when the FP32 result cannot be trusted to the close-call
// margin: a cylinder hit or miss whose discriminant is small against the
// terms it cancels (near-tangent rays amplify FP32 rounding by 1/sqrt(disc)).
constexpr float ILL_DISC = 1e-3f;

// Error estimates of the FP32 distances: the magnitudes that meet in a
// candidate's formula times a rounding scale, over the formula's
// denominator.  A plane's (g - x) / u, with g and x each rounded once to FP32
// and one rounding per operation, is off by at most 2^-24 (|g| + |x|) / |u|
// plus a few ulp of t: F32_ERR (2^-23) is twice that.  A cylinder's root
// moves by about (|dc| + 2 t |db|) / (2 sqrt(disc)) for errors dc, db of the
// quadratic's terms: F32_ERR_CYL (2^-22) times their magnitudes.
constexpr float F32_ERR = 0x1p-23f;
constexpr float F32_ERR_CYL = 0x1p-22f;
// Largest estimated error of the FP32 winner, relative to max(1 cm, d),
// before the flight is redone in FP64 (below the variant's 1e-5 bar).
constexpr float F32_ERR_MAX = 8e-6f;


__device__ __forceinline__ float surface_distance_f(const DevGeom& g, int s, int type, int side, bool on, float x,
                                                    float y, float z, const DirF& d, bool& ill, float& err) {
    const float4 c = __ldg(g.s_coeff + s);
    float t;
    if (type <= S_PZ) {
        if (on) return FINF;
        const float dd = type == S_PX ? d.u : (type == S_PY ? d.v : d.w);
        if (!(side > 0 ? dd < 0.f : dd > 0.f)) return FINF;
        const float xx = type == S_PX ? x : (type == S_PY ? y : z);
        const float ii = type == S_PX ? d.iu : (type == S_PY ? d.iv : d.iw);
        t = (c.x - xx) * ii;
        err = F32_ERR * (fabsf(c.x) + fabsf(xx)) * fabsf(ii);
    } else if (type == S_P) {
        if (on) return FINF;
        const float den = (c.x * d.u + c.y * d.v) + c.z * d.w;
        if (!(side > 0 ? den < 0.f : den > 0.f)) return FINF;
        t = (c.w - ((c.x * x + c.y * y) + c.z * z)) / den;
        err = F32_ERR * (((fabsf(c.x * x) + fabsf(c.y * y)) + fabsf(c.z * z)) + fabsf(c.w)) / fabsf(den);
    } else {
        const float qx = x - c.x, qy = y - c.y;
        const float a = d.u * d.u + d.v * d.v;
        const float b = qx * d.u + qy * d.v;
        // the quadratic's terms carry rounding of their size: t moves by
        // about (|dc| + 2 t |db|) / (2 sqrt(disc)), near-tangent rays (small
        // disc) and large frames (big q, r) blowing it up
        const float bsz = fabsf(qx * d.u) + fabsf(qy * d.v);
        const float csz = (qx * qx + qy * qy) + c.z;
        if (on) {
            if (side < 0 && b < 0.f) t = (-2.0f * b) / a;
            else return FINF;
            err = F32_ERR_CYL * 2.0f * bsz / a;
        } else {
            const float cc = (qx * qx + qy * qy) - c.z;
            if (a == 0.f) return FINF;
            const float bb = b * b, ac = a * cc;
            const float disc = bb - ac;
            if (fabsf(disc) <= ILL_DISC * (bb + fabsf(ac)) && (side < 0 || b < 0.f)) ill = true;
            if (disc <= 0.f) return FINF;
            const float sq = sqrtf(disc);
            if (side < 0) t = (b <= 0.f) ? (-b + sq) / a : -cc / (b + sq);
            else {
                if (!(b < 0.f)) return FINF;
                t = cc / (-b + sq);
            }
            err = F32_ERR_CYL * (csz + 2.0f * fabsf(t) * bsz) / (2.0f * sq) + F32_ERR_CYL * fabsf(t);
        }
    }
    return t < 0.f ? 0.f : t;
}

struct Best2 {
    float d1, d2, e1, e2;   // the two smallest distances and their error estimates
    bool ill;
    Hit h;
    __device__ __forceinline__ void offer(float t, float err, int level, int surf, int side, int dim, int dsign,
                                          int entry) {
        if (t < d1) {
            d2 = d1; e2 = e1; d1 = t; e1 = err;
            h.level = level; h.surf = surf; h.side = side; h.dim = dim; h.dsign = dsign; h.entry = entry;
        } else if (t < d2) {
            d2 = t; e2 = err;
        }
    }
};

template <bool CSG>
__device__ __forceinline__ Best2 distance_f32(const DevGeom& g, const St& s, const DirF& df) {
    Best2 b;
    b.d1 = FINF; b.d2 = FINF; b.e1 = 0.f; b.e2 = 0.f; b.ill = false;
    b.h.d = DINF; b.h.level = -1; b.h.surf = -1; b.h.side = 0; b.h.dim = -1; b.h.dsign = 0; b.h.entry = -1;
    double x = s.x, y = s.y, z = s.z;
    const float d3[3] = {df.u, df.v, df.w};
    const float v3[3] = {df.iu, df.iv, df.iw};
#pragma unroll 1
    for (int l = 0; l < s.nlev; ++l) {
        const Lv L = lv_get(s, l);
        // the next level's frame is this level's element frame: one FP64
        // subtraction chain serves both
        const double xn = x - L.tx, yn = y - L.ty, zn = z - L.tz;
        const int4 ui = __ldg(g.u_info + L.u);
        if (!CSG && ui.w >= 0) {
            const int4 dm = __ldg(g.l_dim + ui.w), of = __ldg(g.l_off + ui.w);
            const int n3[3] = {dm.x, dm.y, dm.z};
            const int o3[3] = {of.x, of.y, of.z};
            const int i3[3] = {L.i, L.j, L.k};
            const float e3[3] = {float(xn), float(yn), float(zn)};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const bool up = d3[d] > 0.f;
                if (!(up ? (i3[d] < n3[d] - 1 || l == 0) : (d3[d] < 0.f && (i3[d] > 0 || l == 0)))) continue;
                const float fo = __ldg((up ? g.l_hif : g.l_lof) + o3[d] + i3[d]);
                const float t = (fo - e3[d]) * v3[d];
                b.offer(t < 0.f ? 0.f : t, F32_ERR * (fabsf(fo) + fabsf(e3[d])) * fabsf(v3[d]), l,
                        -1 - (2 * d + (up ? 1 : 0)), 0, d, up ? 1 : -1, -1);
            }
        } else {
            const int2 rg = __ldg(g.c_range + L.cell);
            int first = rg.x, cnt = rg.y & CS_COUNT_MASK;
            bool by_index = false;
            if (rg.y & CS_SLAB_FLAG) {
                const int4 s0 = __ldg(g.c_slab0 + L.cell), s1 = __ldg(g.c_slab1 + L.cell);
                const int lo3[3] = {s0.x, s0.z, s1.x};
                const int hi3[3] = {s0.y, s0.w, s1.y};
                const float e3[3] = {float(xn), float(yn), float(zn)};
                const float* fs = g.c_slabf + 6 * L.cell;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const bool up = d3[d] > 0.f;
                    const int e = up ? hi3[d] : (d3[d] < 0.f ? lo3[d] : -1);
                    if (e < 0) continue;
                    const int sid = cs_surface(__ldg(g.cs + e));
                    if (s.on_lev == l && s.on_surf == sid) continue;
                    const float fo = __ldg(fs + 2 * d + (up ? 1 : 0));
                    const float t = (fo - e3[d]) * v3[d];
                    b.offer(t < 0.f ? 0.f : t, F32_ERR * (fabsf(fo) + fabsf(e3[d])) * fabsf(v3[d]), l, sid,
                            up ? -1 : 1, -1, 0, e);
                }
                if (rg.y & CS_PAIR_FLAG) {
                    const float xf = float(x), yf = float(y), zf = float(z);
                    const int4 p0 = __ldg(g.c_pair + 2 * L.cell), p1 = __ldg(g.c_pair + 2 * L.cell + 1);
                    const int lo3p[3] = {p0.x, p0.z, p1.x};
                    const int hi3p[3] = {p0.y, p0.w, p1.y};
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        const int ea = lo3p[f] >= 0 ? lo3p[f] : hi3p[f];
                        if (ea < 0) continue;
                        const float4 cf = __ldg(g.s_coeff + cs_surface(__ldg(g.cs + ea)));
                        const float den = (cf.x * df.u + cf.y * df.v) + cf.z * df.w;
                        const int e = den < 0.f ? lo3p[f] : (den > 0.f ? hi3p[f] : -1);
                        if (e < 0) continue;
                        const int sid = cs_surface(__ldg(g.cs + e));
                        if (s.on_lev == l && s.on_surf == sid) continue;
                        const float dw = __ldg(g.s_coeff + sid).w;
                        const float t = (dw - ((cf.x * xf + cf.y * yf) + cf.z * zf)) / den;
                        const float err =
                            F32_ERR * (((fabsf(cf.x * xf) + fabsf(cf.y * yf)) + fabsf(cf.z * zf)) + fabsf(dw)) /
                            fabsf(den);
                        b.offer(t < 0.f ? 0.f : t, err, l, sid, den < 0.f ? 1 : -1, -1, 0, e);
                    }
                }
                const int2 rr = __ldg(g.c_rest + L.cell);
                first = rr.x; cnt = rr.y; by_index = true;
            }
            if (cnt > 0) {
                const float xf = float(x), yf = float(y), zf = float(z);
                for (int k = 0; k < cnt; ++k) {
                    const int ei = by_index ? __ldg(g.rest_e + first + k) : first + k;
                    const int e = __ldg(g.cs + ei);
                    const int sid = cs_surface(e), side = cs_side(e);
                    const bool on = (s.on_lev == l && s.on_surf == sid);
                    float err = 0.f;
                    const float t = surface_distance_f(g, sid, cs_type(e), side, on, xf, yf, zf, df, b.ill, err);
                    b.offer(t, err, l, sid, side, -1, 0, ei);
                }
            }
        }
        x = xn; y = yn; z = zn;
    }
    // the winner must be accurate to F32_ERR_MAX and certainly ahead of the
    // runner-up; else the caller redoes the flight in FP64
    if (b.d1 < FINF && (b.e1 > F32_ERR_MAX * fmaxf(1.0f, b.d1) || b.d2 - b.d1 <= b.e1 + b.e2)) b.ill = true;
    b.h.d = double(b.d1);
    return b;
}

__device__ __forceinline__ bool close_call(float a, float b) {
    return fabsf(a - b) <= CLOSE_REL * fmaxf(fmaxf(a, b) < FINF ? fmaxf(a, b) : 1.0f, 1.0f);
}

enum { CR_OK = 0, CR_REFLECT = 1, CR_ESCAPE = 2, CR_LOST = 3, CR_FIND = 4, CR_ENTER = 5 };

__device__ __forceinline__ void reflect_plane(const DevGeom& g, St& s, int sid, int dim) {
    int type = dim;
    if (sid >= 0) type = __ldg(g.s_info + sid) & 15;
    if (type == S_PX) s.d.u = -s.d.u;
    else if (type == S_PY) s.d.v = -s.d.v;
    else if (type == S_PZ) s.d.w = -s.d.w;
    else {
        double c0, c1, c2, c3;
        load_coef(g, sid, c0, c1, c2, c3);
        const double nd = (c0 * s.d.u + c1 * s.d.v) + c2 * s.d.w;
        const double nn = (c0 * c0 + c1 * c1) + c2 * c2;
        const double k = (2.0 * nd) / nn;
        s.d.u = s.d.u - k * c0;
        s.d.v = s.d.v - k * c1;
        s.d.w = s.d.w - k * c2;
    }
    set_inverse(s.d);
}

// Alg. 4 with face adjacency: the cells on the far side of the crossed face
// (precomputed from box overlap) are tried first; if none holds the point
// the whole universe is searched.  In a geometry whose cells partition space
// the holding cell is unique, so the result equals the linear scan's.
__device__ __forceinline__ int csg_cross_search(const DevGeom& g, int u, int cell, const Pt& p, int xs, int xsn,
                                                int entry) {
    if (entry >= 0) {
        const int2 adj = __ldg(g.cs_adj + entry);
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
            const int cand = k == 0 ? adj.x : adj.y;
            if (cand >= 0 && cell_holds(g, cand, p, xs, xsn)) return cand;
        }
    }
    return csg_search(g, u, p, cell, xs, xsn);
}

// cross_surface in one rect array level (Alg. 6): the neighbouring element,
// or at the root's outer face its boundary condition.  Returns CR_ENTER
// with the element's daughter in dau, or a final result.
__device__ __forceinline__ int cross_level_rect(const DevGeom& g, St& s, int l, Lv& L, int lat, const Hit& h, int& dau) {
    int ijk[3] = {L.i, L.j, L.k};
    const int4 dm = __ldg(g.l_dim + lat);
    const int n3[3] = {dm.x, dm.y, dm.z};
    int ni = 0, nn = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d == h.dim) { ijk[d] += h.dsign; ni = ijk[d]; nn = n3[d]; }
    if (ni < 0 || ni >= nn) {
        if (l != 0) return CR_LOST;
        const int bc = (dm.w >> (2 * (2 * h.dim + (h.dsign > 0)))) & 3;
        if (bc == BC_REFLECT) { reflect_plane(g, s, -1, h.dim); return CR_REFLECT; }
        return CR_ESCAPE;
    }
    dau = enter_element(g, L, lat, ijk[0], ijk[1], ijk[2]);
    return CR_ENTER;
}

// cross_surface in one CSG level (Alg. 4): the cell on the other side of the
// crossed surface, or at the root its boundary condition.
__device__ __forceinline__ int cross_level_csg(const DevGeom& g, St& s, int l, Lv& L, const Hit& h, int& dau) {
    double x, y, z;
    local_at(s, l, x, y, z);
    const Pt p = make_pt(x, y, z);
    const int c = csg_cross_search(g, L.u, L.cell, p, h.surf, -h.side, h.entry);
    if (c < 0) {
        if (l != 0) return CR_LOST;
        const int bc = (__ldg(g.s_info + h.surf) >> 4) & 3;
        if (bc == BC_REFLECT) { reflect_plane(g, s, h.surf, -1); return CR_REFLECT; }
        return CR_ESCAPE;
    }
    dau = enter_cell(g, L, c);
    return CR_ENTER;
}

__device__ __forceinline__ int dp_cross(const Tracker* t, const DevGeom& g, St& s, int l, Lv& L, int lat, const Hit& h,
                                        int& dau);

// Alg. 8 at the hit's level (Alg. 4 for CSG, Alg. 6 for rect).  Returns
// CR_FIND when the levels below the crossing must be found again (the
// caller runs find_from(find_level)), else a final result.
template <int TK>
__device__ __forceinline__ int cross_surface(const DevGeom& g, St& s, const Hit& h, int& find_level) {
    constexpr bool CSG = TK == TK_CSG;
    find_level = -1;
    const int l = h.level;
    if (l < 0 || l >= MAXL) return CR_LOST;
    Lv L = lv_get(s, l);
    const int4 ui = __ldg(g.u_info + L.u);
    s.on_lev = l;
    s.on_surf = h.surf;
    int dau = 0, cr;
    if constexpr (TK == TK_DP) cr = dp_cross(get_tracker(g, ui), g, s, l, L, ui.w, h, dau);
    else if (!CSG && ui.w >= 0) cr = cross_level_rect(g, s, l, L, ui.w, h, dau);
    else cr = cross_level_csg(g, s, l, L, h, dau);
    if (cr != CR_ENTER) return cr;
    lv_set(s, l, L);
    if (dau < 0) {
        s.nlev = l + 1;
        s.mat = ~dau;
        return CR_OK;
    }
    if (l + 1 < MAXL) lv_set_u(s, l + 1, dau);
    find_level = l + 1;
    return CR_FIND;
}

// ---------------------------------------------------------------------------
// Dynamic polymorphism (the paper's DP method, Sec. 4.1): a tracker base
// class with the per-universe operations of Table 1 as virtual methods, a
// rect array tracker and a CSG tracker deriving from it, and get_tracker
// returning the object for a universe's type.  The objects live in the
// geometry's device memory (built there by a kernel, since their virtual
// table pointers must be device addresses); the tracking kernels only see
// base pointers, so every per-level operation is an indirect call.
// ---------------------------------------------------------------------------
struct Tracker {
    __device__ virtual bool find(const DevGeom&, Lv&, int, const Pt&, bool, int&) const { return false; }
    __device__ virtual void distance(const DevGeom&, const St&, int, const Lv&, int, double, double, double, long long,
                                     double, Hit&, long long&) const {}
    __device__ virtual int cross(const DevGeom&, St&, int, Lv&, int, const Hit&, int&) const { return CR_LOST; }
};

struct RectTracker final : Tracker {
    __device__ bool find(const DevGeom& g, Lv& L, int lat, const Pt& p, bool root, int& dau) const override {
        return find_level_rect(g, L, lat, p, root, dau);
    }
    __device__ void distance(const DevGeom& g, const St& s, int l, const Lv& L, int lat, double x, double y, double z,
                             long long, double, Hit& c, long long& ck) const override {
        dist_level_rect(g, s, l, L, lat, x, y, z, c, ck);
    }
    __device__ int cross(const DevGeom& g, St& s, int l, Lv& L, int lat, const Hit& h, int& dau) const override {
        return cross_level_rect(g, s, l, L, lat, h, dau);
    }
};

struct CsgTracker final : Tracker {
    __device__ bool find(const DevGeom& g, Lv& L, int, const Pt& p, bool, int& dau) const override {
        return find_level_csg(g, L, -1, p, dau);
    }
    __device__ void distance(const DevGeom& g, const St& s, int l, const Lv& L, int, double x, double y, double z,
                             long long hk, double hd, Hit& c, long long& ck) const override {
        dist_level_csg(g, s, l, L, x, y, z, hk, hd, c, ck);
    }
    __device__ int cross(const DevGeom& g, St& s, int l, Lv& L, int, const Hit& h, int& dau) const override {
        return cross_level_csg(g, s, l, L, h, dau);
    }
};

// The objects in the geometry's DP region: the table of base pointers
// (index 0 rect arrays, 1 CSG universes, hex arrays included), then the objects.
struct DpTable {
    const Tracker* t[2];
    alignas(16) unsigned char rect[16];
    alignas(16) unsigned char csg[16];
};
static_assert(sizeof(RectTracker) <= 16 && sizeof(CsgTracker) <= 16, "tracker objects exceed their slots");
static_assert(sizeof(DpTable) <= TRK_DP_BYTES, "DP region too small");

__device__ __forceinline__ const Tracker* get_tracker(const DevGeom& g, const int4& ui) {
    return static_cast<const DpTable*>(g.dp)->t[ui.w >= 0 ? 0 : 1];
}
__device__ __forceinline__ bool dp_find(const Tracker* t, const DevGeom& g, Lv& L, int lat, const Pt& p, bool root,
                                        int& dau) {
    return t->find(g, L, lat, p, root, dau);
}
__device__ __forceinline__ void dp_distance(const Tracker* t, const DevGeom& g, const St& s, int l, const Lv& L, int lat,
                                            double x, double y, double z, long long hk, double hd, Hit& c,
                                            long long& ck) {
    t->distance(g, s, l, L, lat, x, y, z, hk, hd, c, ck);
}
__device__ __forceinline__ int dp_cross(const Tracker* t, const DevGeom& g, St& s, int l, Lv& L, int lat, const Hit& h,
                                        int& dau) {
    return t->cross(g, s, l, L, lat, h, dau);
}

// ---------------------------------------------------------------------------
// Run parameters and per-thread counters
// ---------------------------------------------------------------------------
struct RunP {
    uint64_t first_id;
    uint64_t max_segments;
    double p_absorb;
    double max_path;
    uint32_t seed_lo;
    int trace_cap;
    unsigned long long* mesh;   // mesh track-length tally (F_MESH)
    // power iteration (F_FISS): the previous cycle's k, per-history fission
    // outputs, the cycle's nu sum
    const double* knorm;
    double* fis_pos;            // 3 per history
    int* fis_n;                 // sites per history
    unsigned long long* nu_sum;
    // segment log of the event kernel (F_TRACE): trace_cap entries per particle
    int* tr_inst = nullptr;
    double* tr_len = nullptr;
};

// Per-thread event counts (32-bit: one thread tracks far fewer than 2^32
// segments), reduced over the warp and added once per warp at kernel end.
constexpr int NCOUNT = 11;
struct Counts {
    unsigned k[NCOUNT];
};

__device__ __forceinline__ void flush_counts(Counts& c, unsigned long long* out) {
#pragma unroll
    for (int i = 0; i < NCOUNT; ++i) {
        unsigned long long v = c.k[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(out + i, v);
    }
}

__device__ __forceinline__ void kernel_status(unsigned long long* cnt, int st) {
    atomicCAS(cnt + TRK_K_STATUS, 0ULL, (unsigned long long)(long long)st);
}

enum { F_REC = 1, F_CUT = 2, F_TRACE = 4, F_MESH = 8, F_FISS = 16 };

// Mesh index per axis: the largest i in -1..n with g_i <= x (-1 and n are the
// two sides outside the mesh), by order keys; the start guess from the
// planes' span only saves steps, the key compares decide.
__device__ __forceinline__ int mesh_index(const DevGeom& g, int d, double x, long long kx) {
    const int n = g.m_n[d];
    const long long* key = g.m_key + g.m_go[d];
    double e = floor((x - g.m_lo[d]) * g.m_inv[d]);
    int i = e < -1.0 ? -1 : (e > double(n) ? n : int(e));
    while (i >= 0 && __ldg(key + i) > kx) --i;
    while (i < n && __ldg(key + i + 1) <= kx) ++i;
    return i;
}

// Superimposed mesh track-length tally of one segment (start s.x, s.y, s.z,
// length len along the direction): from the start, per axis the next mesh
// plane in the direction of flight (none beyond the outermost) at
// t = (g - x0) * (1/u); a piece ends at the smallest t below len (x before y
// before z on ties), a t below the piece's start counts as the start; pieces
// inside the mesh add llrint(length * 2^32) to their bin (x fastest).
__device__ __forceinline__ void mesh_walk(const DevGeom& g, const St& s, double len, unsigned long long* mesh) {
    const double p3[3] = {s.x, s.y, s.z};
    const double d3[3] = {s.d.u, s.d.v, s.d.w};
    const double v3[3] = {s.d.iu, s.d.iv, s.d.iw};
    int idx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) idx[d] = mesh_index(g, d, p3[d], okey(p3[d]));
    double t0 = 0.0;
    for (;;) {
        double tn = len;
        long long kn = okey(len);
        int ax = -1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int pl = -1;
            if (d_gt0(d3[d]) && idx[d] < g.m_n[d]) pl = idx[d] + 1;
            else if (d_lt0(d3[d]) && idx[d] >= 0) pl = idx[d];
            if (pl < 0) continue;
            const double t = (__ldg(g.m_grid + g.m_go[d] + pl) - p3[d]) * v3[d];
            const long long kt = okey(t);
            if (kt < kn) { tn = t; kn = kt; ax = d; }
        }
        if (kn < okey(t0)) tn = t0;
        if (idx[0] >= 0 && idx[0] < g.m_n[0] && idx[1] >= 0 && idx[1] < g.m_n[1] && idx[2] >= 0 && idx[2] < g.m_n[2]) {
            const long long b = idx[0] + (long long)g.m_n[0] * (idx[1] + (long long)g.m_n[1] * idx[2]);
            atomicAdd(mesh + b, (unsigned long long)__double2ll_rn((tn - t0) * 4294967296.0));
        }
        if (ax < 0) break;
        t0 = tn;
        idx[ax] += d_gt0(ax == 0 ? d3[0] : (ax == 1 ? d3[1] : d3[2])) ? 1 : -1;
    }
}


// ---------------------------------------------------------------------------
// Power iteration (Alg. 1) with a synthetic fission source: an absorption in
// a material with nu > 0 banks floor(nu / k + xi) sites (at most
// FISSION_MAX) at the absorption point, k the previous cycle's estimate
// (*rp.knorm) and xi the first value of counter (pid, e, TAG_FISSION, 0), e
// the absorbing collision's event number; the cycle's nu sum gains
// llrint(nu * 2^32).  Returns the site count.
constexpr int FISSION_MAX = 8;

__device__ __forceinline__ int fission_sites(const DevGeom& g, uint32_t pid, uint32_t event, int mat, const RunP& rp) {
    const double nu = __ldg(g.nu + mat);
    const double k = *rp.knorm;
    if (!d_gt0(k) || !d_gt0(nu)) return 0;
    double xf, unused;
    uniform2(pid, event, TAG_FISSION, 0, rp.seed_lo, uint32_t(g.gid), xf, unused);
    const double ns = floor(nu / k + xf);
    atomicAdd(rp.nu_sum, (unsigned long long)__double2ll_rn(nu * 4294967296.0));
    return d_lt(ns, double(FISSION_MAX)) ? int(ns) : FISSION_MAX;
}

__device__ __forceinline__ void fission_out(const RunP& rp, long long i, int ns, double x, double y, double z) {
    rp.fis_n[i] = ns;
    if (ns > 0) { rp.fis_pos[3 * i] = x; rp.fis_pos[3 * i + 1] = y; rp.fis_pos[3 * i + 2] = z; }
}

// ---------------------------------------------------------------------------
// One history as three steps (shared by the history and event kernels).
// Alg. 2 with the synthetic physics:
//   dc = tau / Sigma (Sigma = 0: +inf); if d < dc: tally(d); r += d Omega;
//   tau -= Sigma d; cross; else: tally(dc); r += dc Omega; collide.
// tally adds llrint(len * 2^32) to the leaf instance's bin.  Collision e
// (1-based) draws (xi_abs, xi_tau) from counter (pid, e, TAG_SCALARS, 0):
// absorbed iff xi_abs < p_a, else a new isotropic direction at event e and
// tau = -log(xi_tau); the on-surface state is cleared.  A history stops
// after max_segments segments.
// ---------------------------------------------------------------------------
struct Ctx {
    uint32_t pid, event;
    long long nseg;
    double path;
    uint64_t hash;
    int status;
};

// A_REDO: an FP32-local flight that must be redone in FP64, left untouched
// for the caller to queue (the event kernels redo such flights together, in
// full warps, after the flight pass).
enum { A_CROSS = 0, A_COLLIDE = 1, A_FLY = 2, A_DONE = 3, A_REDO = 4 };

template <int TK, int FLAGS>
__device__ __forceinline__ int step_flight(const DevGeom& g, St& s, Hit& h, Ctx& c, const RunP& rp,
                                           unsigned long long* __restrict__ tally, Counts& cnt,
                                           int* __restrict__ tr_inst, double* __restrict__ tr_len, long long i) {
    h = distance_to_boundary<TK>(g, s);
    const double sig = __ldg(g.sigma + s.mat);
#if defined(TRK_EXACT) || !TRK_FAST_RSIGMA
    const double dc = d_gt0(sig) ? s.tau / sig : DINF;
#else
    // fast build: tau times the material's reciprocal cross section, within
    // an ulp of the quotient, without the division's instruction sequence
    const double dc = d_gt0(sig) ? s.tau * __ldg(g.rsigma + s.mat) : DINF;
#endif
    const bool crossing = d_lt(h.d, dc);
    double len = crossing ? h.d : dc;
    if (!d_finite_lt_inf(len)) { c.status = TRK_E_LOST; cnt.k[TRK_K_LOST]++; return A_DONE; }
    const int inst = instance(s);
    bool stop_cut = false;
    if (FLAGS & F_CUT) {
        if (!d_lt(c.path + len, rp.max_path)) { len = rp.max_path - c.path; stop_cut = true; }
        else c.path = c.path + len;
    }
    const long long q = __double2ll_rn(len * 4294967296.0);
    atomicAdd(tally + inst, (unsigned long long)q);
    if (FLAGS & F_MESH) mesh_walk(g, s, len, rp.mesh);
    if (FLAGS & F_REC) c.hash = fnv(fnv(c.hash, uint64_t(int64_t(inst))), uint64_t(dbits(len)));
    if (FLAGS & F_TRACE) {
        if (c.nseg < rp.trace_cap) {
            tr_inst[i * rp.trace_cap + c.nseg] = inst;
            tr_len[i * rp.trace_cap + c.nseg] = len;
        }
    }
    s.x = s.x + len * s.d.u;
    s.y = s.y + len * s.d.v;
    s.z = s.z + len * s.d.w;
    c.nseg++;
    cnt.k[TRK_K_SEGMENTS]++;
    if (stop_cut) { c.status = TRK_P_CUTOFF; cnt.k[TRK_K_CUTOFF]++; return A_DONE; }
    if (crossing) {
        s.tau = s.tau - sig * h.d;
        cnt.k[TRK_K_CROSSINGS]++;
        return A_CROSS;
    }
    return A_COLLIDE;
}

// Length of an FP32-local crossing.  A plane crossing is re-evaluated in
// FP64 from the FP64 frame coordinates (the same arithmetic as the FP64
// path), so the particle lands on the plane and the array and universe
// searches that follow see what they would in FP64 (exact = true).  Cylinder
// crossings keep the FP32 length: only small linear cell scans follow them.
__device__ __forceinline__ double f32_crossing_length(const DevGeom& g, const St& s, const Best2& b, bool& exact) {
    const Hit& h = b.h;
    // FP64 coordinates of the winner's level frame (the chain the scan took)
    double wx, wy, wz;
    local_at(s, h.level, wx, wy, wz);
    double t = 0.0;
    bool plane = false;
    if (h.surf < 0) {
        int lat = 0, idx = 0;
#pragma unroll
        for (int l = 0; l < MAXL; ++l)
            if (l == h.level) {
                lat = __ldg(g.u_info + s.lv[l].u).w;
                idx = h.dim == 0 ? s.lv[l].i : (h.dim == 1 ? s.lv[l].j : s.lv[l].k);
            }
        const int4 of = __ldg(g.l_off + lat);
        const int go = h.dim == 0 ? of.x : (h.dim == 1 ? of.y : of.z);
        const double gv = __ldg(g.l_grid + go + idx + (h.dsign > 0 ? 1 : 0));
        const double pv = h.dim == 0 ? wx : (h.dim == 1 ? wy : wz);
        const double iv = h.dim == 0 ? s.d.iu : (h.dim == 1 ? s.d.iv : s.d.iw);
        t = (gv - pv) * iv;
        plane = true;
    } else {
        const int type = __ldg(g.s_info + h.surf) & 15;
        if (type <= S_PZ) {
            const double gv = __ldg(g.s_coef + 4 * h.surf);
            const double pv = type == S_PX ? wx : (type == S_PY ? wy : wz);
            const double iv = type == S_PX ? s.d.iu : (type == S_PY ? s.d.iv : s.d.iw);
            t = (gv - pv) * iv;
            plane = true;
        } else if (type == S_P) {
            t = surface_distance(g, h.surf, type, h.side, false, wx, wy, wz, s.d);
            plane = true;
        }
    }
    exact = plane;
    if (!plane) return double(b.d1);
    return d_lt0(t) ? 0.0 : t;
}

// The FP64 flight as a call, for the FP32-local flight's close calls (a
// fraction of a percent of the flights): inlined there it would double the
// FP32 kernel's code and registers.
template <bool CSG, int FLAGS>
static __device__ __noinline__ int step_flight_fp64_call(const DevGeom& g, St& s, Hit& h, Ctx& c, const RunP& rp,
                                                         unsigned long long* __restrict__ tally, Counts& cnt,
                                                         int* __restrict__ tr_inst, double* __restrict__ tr_len,
                                                         long long i) {
    return step_flight<CSG, FLAGS>(g, s, h, c, rp, tally, cnt, tr_inst, tr_len, i);
}

// FP32-local flight: distances and the flight decision in FP32, position
// and tau in FP64; close calls are redone by the FP64 step, at once or (DEFER)
// by the caller after A_REDO, with nothing of the particle changed.
template <bool CSG, int FLAGS, bool DEFER = false>
__device__ __forceinline__ int step_flight_f32(const DevGeom& g, St& s, Hit& h, Ctx& c, const RunP& rp,
                                               unsigned long long* __restrict__ tally, Counts& cnt,
                                               int* __restrict__ tr_inst, double* __restrict__ tr_len, long long i) {
    const DirF df = dir_f32(s.d);
    const Best2 b = distance_f32<CSG>(g, s, df);
    const double sig = __ldg(g.sigma + s.mat);
    const float sigf = float(sig);
    const float dcf = sigf > 0.f ? float(s.tau) / sigf : FINF;
    if (b.ill || close_call(b.d1, b.d2) || close_call(b.d1, dcf) || !(fminf(b.d1, dcf) < FINF)) {
        cnt.k[TRK_K_CLOSE_CALLS]++;
        if (DEFER) return A_REDO;
        return step_flight_fp64_call<CSG, FLAGS>(g, s, h, c, rp, tally, cnt, tr_inst, tr_len, i);
    }
    h = b.h;
    const bool crossing = b.d1 < dcf;
    const float lenf = crossing ? b.d1 : dcf;
    double len = double(lenf);
    bool exact_len = false;
    if (crossing) len = f32_crossing_length(g, s, b, exact_len);
    const int inst = instance(s);
    bool stop_cut = false;
    if (FLAGS & F_CUT) {
        if (!d_lt(c.path + len, rp.max_path)) { len = rp.max_path - c.path; stop_cut = true; }
        else c.path = c.path + len;
    }
    const unsigned long long q = (stop_cut || exact_len) ? (unsigned long long)__double2ll_rn(len * 4294967296.0)
                                                        : __float2ull_rn(lenf * 4294967296.0f);
    atomicAdd(tally + inst, q);
    if (FLAGS & F_REC) c.hash = fnv(fnv(c.hash, uint64_t(int64_t(inst))), uint64_t(dbits(len)));
    if (FLAGS & F_TRACE) {
        if (c.nseg < rp.trace_cap) {
            tr_inst[i * rp.trace_cap + c.nseg] = inst;
            tr_len[i * rp.trace_cap + c.nseg] = len;
        }
    }
    s.x = s.x + len * s.d.u;
    s.y = s.y + len * s.d.v;
    s.z = s.z + len * s.d.w;
    c.nseg++;
    cnt.k[TRK_K_SEGMENTS]++;
    if (stop_cut) { c.status = TRK_P_CUTOFF; cnt.k[TRK_K_CUTOFF]++; return A_DONE; }
    if (crossing) {
        s.tau = s.tau - sig * len;
        cnt.k[TRK_K_CROSSINGS]++;
        return A_CROSS;
    }
    return A_COLLIDE;
}

template <int TK, bool F32, int FLAGS, bool DEFER = false>
__device__ __forceinline__ int step_fly(const DevGeom& g, St& s, Hit& h, Ctx& c, const RunP& rp,
                                        unsigned long long* __restrict__ tally, Counts& cnt,
                                        int* __restrict__ tr_inst, double* __restrict__ tr_len, long long i) {
    static_assert(!(F32 && TK == TK_DP), "the DP tracker is FP64 only");
    if constexpr (F32)
        return step_flight_f32<TK == TK_CSG, FLAGS, DEFER>(g, s, h, c, rp, tally, cnt, tr_inst, tr_len, i);
    else return step_flight<TK, FLAGS>(g, s, h, c, rp, tally, cnt, tr_inst, tr_len, i);
}

__device__ __forceinline__ int after_step(Ctx& c, const RunP& rp, Counts& cnt) {
    if (uint64_t(c.nseg) >= rp.max_segments) { c.status = TRK_E_MAX_SEGMENTS; cnt.k[TRK_K_MAXSEG]++; return A_DONE; }
    return A_FLY;
}

template <int TK>
__device__ TRK_CROSS_INLINE int step_cross(const DevGeom& g, St& s, const Hit& h, Ctx& c, const RunP& rp, Counts& cnt) {
    int fl;
    int cr = cross_surface<TK>(g, s, h, fl);
    if (cr == CR_FIND) cr = find_from<TK>(g, s, fl) == 0 ? CR_OK : CR_LOST;
    if (cr == CR_ESCAPE) { c.status = TRK_P_ESCAPED; cnt.k[TRK_K_ESCAPED]++; return A_DONE; }
    if (cr == CR_LOST) { c.status = TRK_E_LOST; cnt.k[TRK_K_LOST]++; return A_DONE; }
    if (cr == CR_REFLECT) cnt.k[TRK_K_REFLECTIONS]++;
    return after_step(c, rp, cnt);
}

static __device__ TRK_COLLIDE_INLINE int step_collide(const DevGeom& g, St& s, Ctx& c, const RunP& rp, Counts& cnt) {
    const uint32_t gid = uint32_t(g.gid);
    ++c.event;
    cnt.k[TRK_K_COLLISIONS]++;
    double xa, xt;
    uniform2(c.pid, c.event, TAG_SCALARS, 0, rp.seed_lo, gid, xa, xt);
    if (d_lt(xa, rp.p_absorb)) { c.status = TRK_P_ABSORBED; cnt.k[TRK_K_ABSORBED]++; return A_DONE; }
    if (!isotropic(c.pid, c.event, rp.seed_lo, gid, s.d.u, s.d.v, s.d.w)) {
        c.status = TRK_E_LOST; cnt.k[TRK_K_LOST]++; return A_DONE;
    }
    set_inverse(s.d);
    s.tau = -own_log(xt);
    s.on_lev = -1;
    s.on_surf = -1;
    return after_step(c, rp, cnt);
}

// Birth: state from source_init's buffer, then find_cell from the root.
__device__ __forceinline__ bool load_birth(const DevGeom& g, const ParticlesView& P, long long i, St& s) {
    clear_levels(s);
    s.x = P.x[i]; s.y = P.y[i]; s.z = P.z[i];
    s.d.u = P.u[i]; s.d.v = P.v[i]; s.d.w = P.w[i];
    s.tau = P.tau[i];
    set_inverse(s.d);
    s.lv[0].u = g.root;
    return true;
}

}  // namespace dev
}  // namespace trk
