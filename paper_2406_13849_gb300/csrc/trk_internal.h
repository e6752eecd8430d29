// trk_internal.h - flattened device geometry shared by the host builder
// (geometry_build.cpp) and the kernels (trk_kernels.cu).  Not part of the ABI.
//
// Everything a tracker reads lives in one caller-owned device buffer as a
// structure of arrays; DevGeom holds typed pointers into it and is passed to
// every kernel by value.  Two views of the same universes coexist so that one
// handle serves both trackers:
//   CSG view   every universe is a list of CSG cells; array universes appear
//              as pseudo-arrays (Sec. 4.3), one plane-bounded cell per element,
//              searched through a BVH over cell boxes.
//   rect view  rect array universes keep their grid planes (Alg. 5/6).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __CUDACC__
#define TRK_HD_INLINE __host__ __device__ __forceinline__
#else
#define TRK_HD_INLINE inline
#endif

namespace trk {

enum SurfType { S_PX = 0, S_PY = 1, S_PZ = 2, S_P = 3, S_CZ = 4 };
enum Bc { BC_NONE = 0, BC_VACUUM = 1, BC_REFLECT = 2 };

// Compiled nesting depth of the trackers' register-resident level stack.
constexpr int MAXL = 4;
// Cells per BVH leaf at most.
constexpr int BVH_LEAF_MAX = 4;
// Universes with at most this many cells are scanned linearly (Alg. 3).
constexpr int LINEAR_MAX = 4;

// BVH node holding both children's boxes (FP32, rounded outward from padded
// FP64 cell boxes), so one node load tests both children.  A child reference
// >= 0 is an internal node; < 0 is a leaf, -1 - ((first leaf slot << 4) |
// count).  Children are laid out left before right (preorder), and a point
// query walks left before right, so the first holding cell is that of the
// preorder walk.
struct alignas(16) BvhNode {
    float lo0[3], hi0[3];
    float lo1[3], hi1[3];
    int ref0, ref1, pad0, pad1;
};
// Hex lattice for the array tracker's closed-form search: the inverse of
// the lattice-vector matrix (axial q, r from the universe-frame x, y), the
// ring count, the first pseudo-array cell (elements in order: rows
// r = -R..R, q ascending) and the offset of its row-start table in hx_row.
struct alignas(16) HexInfo {
    double i00, i01, i10, i11;
    int rings, first_cell, row, pad;
};

// Bounding interval hierarchy node (Sec. 4.3): along `axis` the left
// child's boxes end at or below clip_l and the right child's start at or
// above clip_r (FP32, rounded outward); the half-spaces may overlap.
// ref0: left child, ref1_axis = ref1 * 4 + axis (references as in BvhNode).
struct alignas(16) BihNode {
    float clip_l, clip_r;
    int ref0, ref1_axis;
};

// Largest BVH depth the builder produces (the walk's stack size).
constexpr int BVH_STACK = 64;

// c_range count field: low bits count, CS_SLAB_FLAG marks a cell with a
// view: at most one lower and one upper axis plane per dimension, up to
// three pairs of general planes with one normal (CS_PAIR_FLAG), and the
// other surfaces as the cell's remaining entries (c_rest / rest_e).
constexpr int CS_SLAB_FLAG = 1 << 30;
// CS_PAIR_FLAG: the view also has plane pairs (c_pair).
constexpr int CS_PAIR_FLAG = 1 << 29;
constexpr int CS_COUNT_MASK = CS_PAIR_FLAG - 1;

// Packed cell-surface entry: (surface << 4) | (type << 1) | (sense > 0).
TRK_HD_INLINE int cs_surface(int e) { return e >> 4; }
TRK_HD_INLINE int cs_type(int e) { return (e >> 1) & 7; }
TRK_HD_INLINE int cs_side(int e) { return (e & 1) ? 1 : -1; }

struct DevGeom {
    // surfaces
    const int* s_info;        // type | (bc << 4) | (rparam+1) << 8 | pscale << 12
    const double* s_coef;     // 4 per surface; px/py/pz: (g,0,0,0); p: (nx,ny,nz,d); cz: (x0,y0,r,r*r)
    const long long* s_key;   // order key of g for px/py/pz (sense tests as integer compares)
    // cells (CSG view)
    const int2* c_range;      // (first, count | CS_SLAB_FLAG) into cs
    const int* cs;            // packed cell-surface entries (see cs_surface / cs_type / cs_side)
    const int2* cs_adj;       // per entry: up to two cells on the far side of that face, -1 none,
                              // (-2,-2) too many (search the BVH directly)
    const int4* c_slab0;      // slab view (CS_SLAB_FLAG cells): entry index of
                              // the lower / upper face on x, y (lo_x, hi_x, lo_y, hi_y), -1 absent
    const int4* c_slab1;      // (lo_z, hi_z, -, -)
    const longlong2* c_slabk; // slab cells, 3 per cell: order keys of the (lower, upper) face per
                              // dimension, LLONG_MIN / LLONG_MAX where absent (containment test)
    const int4* c_slabs;      // slab cells, 2 per cell: surface ids (lo_x, hi_x, lo_y, hi_y),
                              // (lo_z, hi_z, -1, -1); -1 absent
    const int* c_fill;        // >= 0 daughter universe; < 0 material ~fill
    const int2* c_rest;       // slab-view cells: (first, count) into rest_e, the entries that are
                              // not axis planes, in cell order
    const int* rest_e;
    const int4* c_pair;       // view cells, 2 per cell: entries of up to three plane pairs (general
                              // planes with one normal), (lo0, hi0, lo1, hi1), (lo2, hi2, -1, -1);
                              // lo = the "+" entry (left when n.u < 0), hi = the "-" entry
    const int* c_fcls;        // flight class of the cell as a leaf: 0 axis planes only, 1 one
                              // cylinder (inside) and axis planes, 2 one cylinder (outside) and
                              // axis planes, 3 anything else
    const double* c_tr;       // translation into the daughter, 3 per cell
    const int* c_off;         // leaf-instance offset of the cell
    // universes
    const int4* u_info;       // (first cell, cell count, BVH root node or -1, rect lattice >= 0,
                              //  hex lattice -2 - h, or -1)
    const HexInfo* hx;        // hex lattices (array tracker)
    const int* hx_row;        // per hex lattice: first element of row r at hx_row[row + r + rings]
    // rect arrays (rect view)
    const int4* l_dim;        // (nx, ny, nz, packed bc: 2 bits per face xlo..zhi)
    const int4* l_off;        // (x grid offset, y grid offset, z grid offset, element offset)
    const double* l_grid;     // grid planes; dim d of lattice k at l_grid[l_off[k].d]
    const long long* l_gkey;  // order keys of the grid planes, same offsets
    const double* l_ctr;      // element centres (g_i + g_{i+1}) * 0.5, same offsets
    const int* l_fill;        // element universe, at l_fill[l_off[k].w + e]
    const int* l_eoff;        // element instance offset, same indexing
    const int* l_pscale;      // grid planes scale with the pitch (gradient)
    // FP32 copies for the FP32-local precision mode
    const float4* s_coeff;    // px/py/pz: (g,0,0,0); p: (nx,ny,nz,d); cz: (x0,y0,r*r,r)
    const float* l_lof;       // face below element i relative to its centre: g_i - c_i, l_grid offsets
    const float* l_hif;       // face above: g_{i+1} - c_i
    const float* c_slabf;     // 6 per cell: slab faces (lo_x, hi_x, lo_y, hi_y, lo_z, hi_z)
                              // relative to the cell's translation
    // superimposed mesh (track-length tally): planes per axis and their order keys
    const double* m_grid;     // axis d at m_grid[m_go[d]], m_n[d] + 1 planes
    const long long* m_key;
    double m_lo[3], m_inv[3]; // first plane and n / (g_n - g_0) per axis (search start only)
    int m_n[3], m_go[3];      // bins and plane offsets per axis; m_n[0] == 0: no mesh
    // BVH nodes (two child boxes per node); BIH nodes and roots per universe
    const BvhNode* nodes;
    const BihNode* bih;
    const int* u_bih;         // BIH root reference per universe (-1: linear scan)
    int accel;                // CSG cell search: 0 BVH, 1 BIH
    const int* leaf_cells;
    // materials
    const double* sigma;
    const double* rsigma;     // 1 / sigma (0 where sigma = 0): the fast build's collision distance
    const double* nu;         // fission yield per material (0: none), power iteration
    const void* dp;           // DP tracker objects (TRK_TRACKER_DP), built on the device by dp_install
    double src_lo[3], src_hi[3];
    int root, n_inst, n_mat, gid, max_depth, n_univ, n_cells, n_surf;
    int rect_ok;              // the array tracker applies (always 1: hex arrays by closed-form search)
};

// Order key of a double: a < b  <=>  okey(a) < okey(b) for non-NaN values,
// with -0 and +0 equal (IEEE).  Lets FP64 comparisons run on the integer pipe.
TRK_HD_INLINE long long okey_bits(long long b) {
    return b < 0 ? -(b & 0x7fffffffffffffffLL) : b;
}

// Particle buffer written by source_init (structure of arrays).
struct ParticlesView {
    const double* x; const double* y; const double* z;
    const double* u; const double* v; const double* w;
    const double* tau; const int* status;
};

// Records the message returned by trk_last_error() and returns `st`.
int set_error(int st, const char* fmt, ...);

}  // namespace trk

// The library-owned host object behind trk_geom_t.
namespace trk {
// Bytes of the geometry's DP region, and the call that builds the DP
// tracker objects there (a kernel on `stream`; returns a cudaError_t).
constexpr size_t TRK_DP_BYTES = 64;
int dp_install(void* dev, void* stream);
}  // namespace trk

struct trk_geom {
    trk::DevGeom dg;
    size_t bytes = 0;
    int64_t n_inst = 0;
    int n_mat = 0, depth = 0, rect_ok = 0;
    int has_hex = 0;          // hex arrays present: TRK_TRACKER_AUTO picks the CSG tracker
    int n_nodes = 0;
    int max_rect_dim = 0;     // most elements along one axis of a rect array
    unsigned magic = 0;
};
constexpr unsigned TRK_GEOM_MAGIC = 0x7472'6b67u;
