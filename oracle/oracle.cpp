// Plain FP64 CPU oracle for nested-universe particle tracking.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
// the CPU-baseline leg of the benchmark may load this library.  It shares no
// code with the CUDA path: its own JSON reader, its own geometry model, its
// own Philox, log and sampling.  It is written for a reader checking it
// against the paper by eye, not for speed: linear scans, no acceleration
// structure, one history at a time.
//
// What it computes (arXiv 2406.13849):
//   run_histories      Alg. 2 with synthetic physics (constant sigma per
//                      material, absorption probability p_a, isotropic
//                      scatter); no fission or energy.
//   find_cell          Alg. 3 (CSG linear scan), Alg. 5 (rect binary search),
//                      Alg. 7 (descend through daughter universes).
//   cross_surface      Alg. 4 (CSG: another cell that holds the point once
//                      the crossed surface's sense is flipped), Alg. 6 (rect:
//                      ijk +/- 1), Alg. 8 (cross at the surface's level, then
//                      find_cell below).
//   distance_to_surface, move_within_cell, change_direction: Table 1.
//   pseudo-array universes (Sec. 4.3): in "csg" mode every array universe
//                      is rewritten as a CSG universe of plane-bounded cells.
//   cell tallies       track length per leaf cell instance (Sec. 7 cell
//                      tallies), summed as 64-bit fixed point.
// Where the paper is silent the oracle takes a fixed reading; each reading is
// marked "Reading:" below and is the same one the CUDA path follows.
//
// Pins: every function here is checked by the -m "not gpu" tests against
// something other than itself (brute force over every leaf instance in the
// global frame, closed-form chords, Cauchy's 4V/S law, track-length volumes,
// the geometric collision-count law, Philox known-answer vectors, std::log).
// Segment counts: on the benchmark's three-level core and on the hex core a
// collision-free history's whole segment sequence is checked against the
// surface crossings of its straight path, and on batch members against
// brute-force cell membership along it; on every configuration, sampled
// whole histories with collisions (and reflections) are re-derived from the
// flight rules and the Philox counters.  The power iteration's first two
// cycles are rebuilt exactly (bank, site choice, births from the bank);
// later cycles repeat that step and are pinned statistically.
//
// Built with -O2 -ffp-contract=off so that no multiply-add is fused: every
// floating-point operation below is one IEEE-754 double operation.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

// ---------------------------------------------------------------------------
// Scalar type.  With ORACLE_COUNT_FLOPS the tracker runs on a counting type
// that tallies every FP64 add/sub, mul, div, sqrt and compare; this gives the
// algorithmic operation count per segment used as the roofline numerator.
// ---------------------------------------------------------------------------
#ifdef ORACLE_COUNT_FLOPS
struct FlopCount { unsigned long long add, mul, div, sqrt, cmp; };
static thread_local FlopCount g_fc = {0, 0, 0, 0, 0};
struct Real {
    double v;
    Real() : v(0) {}
    Real(double x) : v(x) {}
    friend Real operator+(Real a, Real b) { g_fc.add++; return Real(a.v + b.v); }
    friend Real operator-(Real a, Real b) { g_fc.add++; return Real(a.v - b.v); }
    friend Real operator*(Real a, Real b) { g_fc.mul++; return Real(a.v * b.v); }
    friend Real operator/(Real a, Real b) { g_fc.div++; return Real(a.v / b.v); }
    Real operator-() const { return Real(-v); }
    friend bool operator<(Real a, Real b) { g_fc.cmp++; return a.v < b.v; }
    friend bool operator<=(Real a, Real b) { g_fc.cmp++; return a.v <= b.v; }
    friend bool operator>(Real a, Real b) { g_fc.cmp++; return a.v > b.v; }
    friend bool operator>=(Real a, Real b) { g_fc.cmp++; return a.v >= b.v; }
    friend bool operator==(Real a, Real b) { g_fc.cmp++; return a.v == b.v; }
    friend bool operator!=(Real a, Real b) { g_fc.cmp++; return a.v != b.v; }
};
static inline Real rsqrt_(Real a) { g_fc.sqrt++; return Real(std::sqrt(a.v)); }
static inline double dv(Real a) { return a.v; }
#else
typedef double Real;
static inline Real rsqrt_(Real a) { return std::sqrt(a); }
static inline double dv(Real a) { return a; }
#endif

static const double INF = std::numeric_limits<double>::infinity();

// ---------------------------------------------------------------------------
// Minimal JSON reader (objects, arrays, numbers, strings, literals).
// ---------------------------------------------------------------------------
namespace oj {
struct Val {
    enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
    double num = 0;
    bool b = false;
    std::string str;
    std::vector<Val> arr;
    std::vector<std::pair<std::string, Val>> obj;
    const Val* get(const char* k) const {
        for (auto& kv : obj) if (kv.first == k) return &kv.second;
        return nullptr;
    }
};
struct Reader {
    const char* p; const char* e; std::string err;
    void ws() { while (p < e && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p; }
    bool fail(const char* m) { if (err.empty()) err = m; return false; }
    bool parse(Val& v) {
        ws();
        if (p >= e) return fail("unexpected end of JSON");
        char c = *p;
        if (c == '{') {
            v.kind = Val::OBJ; ++p; ws();
            if (p < e && *p == '}') { ++p; return true; }
            for (;;) {
                ws(); Val key;
                if (p >= e || *p != '"' || !parse(key)) return fail("bad object key");
                ws(); if (p >= e || *p != ':') return fail("expected ':'"); ++p;
                Val item; if (!parse(item)) return false;
                v.obj.emplace_back(key.str, std::move(item));
                ws(); if (p < e && *p == ',') { ++p; continue; }
                if (p < e && *p == '}') { ++p; return true; }
                return fail("expected ',' or '}'");
            }
        }
        if (c == '[') {
            v.kind = Val::ARR; ++p; ws();
            if (p < e && *p == ']') { ++p; return true; }
            for (;;) {
                Val item; if (!parse(item)) return false;
                v.arr.push_back(std::move(item));
                ws(); if (p < e && *p == ',') { ++p; continue; }
                if (p < e && *p == ']') { ++p; return true; }
                return fail("expected ',' or ']'");
            }
        }
        if (c == '"') {
            v.kind = Val::STR; ++p;
            while (p < e && *p != '"') {
                if (*p == '\\' && p + 1 < e) { ++p; }
                v.str.push_back(*p++);
            }
            if (p >= e) return fail("unterminated string");
            ++p; return true;
        }
        if (c == 't' && e - p >= 4 && !strncmp(p, "true", 4)) { v.kind = Val::BOOL; v.b = true; p += 4; return true; }
        if (c == 'f' && e - p >= 5 && !strncmp(p, "false", 5)) { v.kind = Val::BOOL; p += 5; return true; }
        if (c == 'n' && e - p >= 4 && !strncmp(p, "null", 4)) { v.kind = Val::NUL; p += 4; return true; }
        // number: copy the token and hand it to strtod (exact round-trip)
        const char* s = p;
        while (p < e && (strchr("+-0123456789.eE", *p) != nullptr)) ++p;
        if (p == s) return fail("unexpected character");
        std::string tok(s, p);
        char* endp = nullptr;
        v.kind = Val::NUM; v.num = strtod(tok.c_str(), &endp);
        if (endp != tok.c_str() + tok.size()) return fail("bad number");
        return true;
    }
};
}  // namespace oj

// ---------------------------------------------------------------------------
// Geometry model (Sec. 1: surfaces, cells as intersections of surface senses,
// universes nested in cells; Sec. 4.3: pseudo-array universes).
// ---------------------------------------------------------------------------
enum SurfType { S_PX = 0, S_PY = 1, S_PZ = 2, S_P = 3, S_CZ = 4 };
enum Bc { BC_NONE = 0, BC_VACUUM = 1, BC_REFLECT = 2 };
enum UType { U_CSG = 0, U_RECT = 1, U_HEX = 2 };

struct Surface {
    int type = 0;
    double c[4] = {0, 0, 0, 0};   // px: g | p: nx ny nz d | cz: x0 y0 r
    int bc = BC_NONE;
    int rparam = -1;               // radius design parameter (transmission gradient)
    int pscale = 0;                // position scales with the lattice pitch
};

struct Cell {
    std::vector<int> surf;         // surface ids, in cell order
    std::vector<int> sense;        // +1 / -1
    int material = -1;
    int daughter = -1;
    double tr[3] = {0, 0, 0};      // translation into the daughter's frame
    long long off = 0;             // first leaf instance below this cell
};

struct Universe {
    int type = U_CSG;
    std::vector<Cell> cells;                 // CSG (and pseudo-array) cells
    std::vector<double> grid[3];             // rect planes per dimension
    int rings = 0;                           // hex
    double a1[2] = {0, 0}, a2[2] = {0, 0}, nrm[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    double half_pitch = 0, z[2] = {0, 0};
    std::vector<int> hq, hr;                 // hex element axial coordinates
    std::vector<int> fill;                   // lattice element fills
    std::vector<long long> eoff;             // lattice element instance offsets
    int bc[6] = {0, 0, 0, 0, 0, 0};          // rect: xlo xhi ylo yhi zlo zhi; hex: side,-,-,-,zlo,zhi
    int pscale = 0;
    long long ninst = -1;
    int n_elem() const {
        if (type == U_RECT) return int((grid[0].size() - 1) * (grid[1].size() - 1) * (grid[2].size() - 1));
        if (type == U_HEX) return int(hq.size());
        return int(cells.size());
    }
};

// Superimposed rectilinear mesh for the track-length tally (the paper's
// "active cycle" flux tally, Sec. 6): increasing plane lists per axis.
struct Mesh {
    std::vector<double> grid[3];
    bool on() const { return !grid[0].empty(); }
    long long bins() const {
        return on() ? (long long)(grid[0].size() - 1) * (long long)(grid[1].size() - 1) * (long long)(grid[2].size() - 1) : 0;
    }
};

struct Geometry {
    Mesh mesh;
    int mode = 0;                  // 0: rect trackers for rect arrays; 1: all-CSG (pseudo-arrays)
    int gid = 0;
    std::vector<double> sigma;
    std::vector<double> nu;        // per material, 0: no fission (power iteration)
    std::vector<Surface> surf;
    std::vector<Universe> univ;
    int root = 0;
    double src[6] = {0, 0, 0, 0, 0, 0};
    int max_depth = 0;
};

static int parse_bc(const oj::Val* v) {
    if (!v || v->kind != oj::Val::STR) return BC_NONE;
    if (v->str == "vacuum") return BC_VACUUM;
    if (v->str == "reflect") return BC_REFLECT;
    return BC_NONE;
}

static bool nums(const oj::Val* v, std::vector<double>& out) {
    if (!v || v->kind != oj::Val::ARR) return false;
    out.clear();
    for (auto& x : v->arr) { if (x.kind != oj::Val::NUM) return false; out.push_back(x.num); }
    return true;
}

// A JSON number holding an integer in [lo, hi] (indices, tags, ring counts).
static bool int_in(const oj::Val* v, double lo, double hi, int& out) {
    if (!v || v->kind != oj::Val::NUM) return false;
    const double x = v->num;
    if (!(x >= lo && x <= hi) || x != std::floor(x)) return false;
    out = int(x);
    return true;
}

static bool finite_all(const std::vector<double>& v) {
    for (double x : v) if (!std::isfinite(x)) return false;
    return true;
}

static long long count_instances(Geometry& g, int u, int depth, std::string& err) {
    if (depth > 16) { err = "universe nesting too deep or cyclic"; return -1; }
    Universe& U = g.univ[u];
    if (U.ninst >= 0) return U.ninst;
    long long total = 0;
    if (U.type == U_CSG) {
        for (auto& c : U.cells) {
            c.off = total;
            if (c.material >= 0) total += 1;
            else {
                long long k = count_instances(g, c.daughter, depth + 1, err);
                if (k < 0) return -1;
                total += k;
            }
        }
    } else {
        U.eoff.assign(U.fill.size(), 0);
        for (size_t e = 0; e < U.fill.size(); ++e) {
            U.eoff[e] = total;
            long long k = count_instances(g, U.fill[e], depth + 1, err);
            if (k < 0) return -1;
            total += k;
        }
    }
    U.ninst = total;
    return total;
}

static int depth_of(const Geometry& g, int u) {
    const Universe& U = g.univ[u];
    int best = 0;
    if (U.type == U_CSG) {
        for (auto& c : U.cells) if (c.daughter >= 0) best = std::max(best, depth_of(g, c.daughter));
    } else {
        for (int f : U.fill) best = std::max(best, depth_of(g, f));
    }
    return best + 1;
}

// Reading: element translation of a rect array element is the centre of its
// box, (g_i + g_{i+1}) * 0.5 per dimension.
static void rect_center(const Universe& U, int i, int j, int k, double* t) {
    t[0] = (U.grid[0][i] + U.grid[0][i + 1]) * 0.5;
    t[1] = (U.grid[1][j] + U.grid[1][j + 1]) * 0.5;
    t[2] = (U.grid[2][k] + U.grid[2][k + 1]) * 0.5;
}

// Reading: hex element (q, r) sits at q*a1 + r*a2 (x, y); its z is the middle
// of the lattice's z range.
static void hex_center(const Universe& U, int e, double* t) {
    double q = U.hq[e], r = U.hr[e];
    t[0] = q * U.a1[0] + r * U.a2[0];
    t[1] = q * U.a1[1] + r * U.a2[1];
    t[2] = (U.z[0] + U.z[1]) * 0.5;
}

// Sec. 4.3: rewrite an array universe as a CSG universe ("pseudo-array").
// Reading: element cells are listed in element order with their faces in the
// order (dim 0 lower, dim 0 upper, dim 1 lower, ...); an outer face of a
// non-root array is left out (its parent level owns that boundary, Sec. 3.2
// "lower-level coincident boundary surfaces are removed"), so border cells
// are unbounded outward; a root array keeps its outer faces with their BC.
static void to_pseudo_array(Geometry& g, int u, bool is_root) {
    Universe& U = g.univ[u];
    std::vector<Cell> cells;
    if (U.type == U_RECT) {
        int n[3];
        std::vector<int> sid[3];
        for (int d = 0; d < 3; ++d) {
            n[d] = int(U.grid[d].size()) - 1;
            for (int i = 0; i <= n[d]; ++i) {
                Surface s;
                s.type = d;  // S_PX, S_PY, S_PZ
                s.c[0] = U.grid[d][i];
                s.pscale = (d < 2) ? U.pscale : 0;
                if (i == 0) s.bc = U.bc[2 * d];
                if (i == n[d]) s.bc = U.bc[2 * d + 1];
                sid[d].push_back(int(g.surf.size()));
                g.surf.push_back(s);
            }
        }
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    Cell c;
                    int ijk[3] = {i, j, k};
                    for (int d = 0; d < 3; ++d) {
                        if (ijk[d] > 0 || is_root) { c.surf.push_back(sid[d][ijk[d]]); c.sense.push_back(+1); }
                        if (ijk[d] < n[d] - 1 || is_root) { c.surf.push_back(sid[d][ijk[d] + 1]); c.sense.push_back(-1); }
                    }
                    int e = i + n[0] * (j + n[1] * k);
                    c.daughter = U.fill[e];
                    c.off = U.eoff[e];
                    rect_center(U, i, j, k, c.tr);
                    cells.push_back(c);
                }
    } else if (U.type == U_HEX) {
        // Face planes of family k are n_k . x = j * h for integer j; the faces
        // of element (q, r) have j = m_k -/+ 1 with m_0 = 2q+r, m_1 = q+2r,
        // m_2 = -q+r.  One surface per (k, j), shared by both neighbours.
        std::map<std::pair<int, int>, int> plane;
        auto get_plane = [&](int fam, int j) {
            auto key = std::make_pair(fam, j);
            auto it = plane.find(key);
            if (it != plane.end()) return it->second;
            Surface s;
            s.type = S_P;
            s.c[0] = U.nrm[fam][0]; s.c[1] = U.nrm[fam][1]; s.c[2] = 0.0;
            s.c[3] = double(j) * U.half_pitch;
            s.bc = U.bc[0];
            int id = int(g.surf.size());
            g.surf.push_back(s);
            plane[key] = id;
            return id;
        };
        int zs[2] = {-1, -1};
        if (is_root) {
            for (int t = 0; t < 2; ++t) {
                Surface s; s.type = S_PZ; s.c[0] = U.z[t]; s.bc = U.bc[4 + t];
                zs[t] = int(g.surf.size()); g.surf.push_back(s);
            }
        }
        std::map<std::pair<int, int>, int> index;
        for (size_t e = 0; e < U.hq.size(); ++e) index[{U.hq[e], U.hr[e]}] = int(e);
        auto has = [&](int q, int r) { return index.count({q, r}) > 0; };
        for (size_t e = 0; e < U.hq.size(); ++e) {
            int q = U.hq[e], r = U.hr[e];
            int m[3] = {2 * q + r, q + 2 * r, -q + r};
            // neighbours on the lower / upper side of each family
            int lo_nb[3][2] = {{q - 1, r}, {q, r - 1}, {q + 1, r - 1}};
            int hi_nb[3][2] = {{q + 1, r}, {q, r + 1}, {q - 1, r + 1}};
            Cell c;
            for (int f = 0; f < 3; ++f) {
                if (is_root || has(lo_nb[f][0], lo_nb[f][1])) { c.surf.push_back(get_plane(f, m[f] - 1)); c.sense.push_back(+1); }
                if (is_root || has(hi_nb[f][0], hi_nb[f][1])) { c.surf.push_back(get_plane(f, m[f] + 1)); c.sense.push_back(-1); }
            }
            if (is_root) {
                c.surf.push_back(zs[0]); c.sense.push_back(+1);
                c.surf.push_back(zs[1]); c.sense.push_back(-1);
            }
            c.daughter = U.fill[e];
            c.off = U.eoff[e];
            hex_center(U, int(e), c.tr);
            cells.push_back(c);
        }
    }
    U.type = U_CSG;
    U.cells = cells;
}

static Geometry* load_geometry(const char* json, size_t len, int mode, std::string& err) {
    oj::Reader rd{json, json + len, ""};
    oj::Val doc;
    if (!rd.parse(doc)) { err = "JSON: " + rd.err; return nullptr; }
    if (doc.kind != oj::Val::OBJ) { err = "description is not an object"; return nullptr; }
    std::unique_ptr<Geometry> g(new Geometry);
    g->mode = mode;
    const oj::Val* v;
    if ((v = doc.get("geometry_id")) && !int_in(v, 0, 2147483647.0, g->gid)) { err = "bad geometry_id"; return nullptr; }
    if (!nums(doc.get("sigma"), g->sigma) || g->sigma.empty()) { err = "missing sigma"; return nullptr; }
    for (double x : g->sigma) if (!(x >= 0.0) || !std::isfinite(x)) { err = "sigma must be finite and >= 0"; return nullptr; }
    g->nu.assign(g->sigma.size(), 0.0);
    if (doc.get("nu")) {
        if (!nums(doc.get("nu"), g->nu) || g->nu.size() != g->sigma.size()) { err = "bad nu"; return nullptr; }
        for (double v : g->nu) if (!(v >= 0.0 && v <= 7.0)) { err = "nu must be in [0, 7]"; return nullptr; }
    }
    v = doc.get("surfaces");
    if (!v || v->kind != oj::Val::ARR) { err = "missing surfaces"; return nullptr; }
    for (auto& sv : v->arr) {
        Surface s;
        const oj::Val* t = sv.get("type");
        std::vector<double> cf;
        if (!t || t->kind != oj::Val::STR || !nums(sv.get("coef"), cf)) { err = "bad surface"; return nullptr; }
        size_t need;
        if (t->str == "px") { s.type = S_PX; need = 1; }
        else if (t->str == "py") { s.type = S_PY; need = 1; }
        else if (t->str == "pz") { s.type = S_PZ; need = 1; }
        else if (t->str == "p") { s.type = S_P; need = 4; }
        else if (t->str == "cz") { s.type = S_CZ; need = 3; }
        else { err = "unknown surface type " + t->str; return nullptr; }
        if (cf.size() != need || !finite_all(cf)) { err = "wrong or non-finite coefficients"; return nullptr; }
        for (size_t i = 0; i < need; ++i) s.c[i] = cf[i];
        s.bc = parse_bc(sv.get("bc"));
        if (s.bc == BC_REFLECT && s.type == S_CZ) { err = "reflecting cylinders are not supported"; return nullptr; }
        // rparam names one of the radius parameters r_0..r_2 of the transmission gradient (-1: none)
        if ((t = sv.get("rparam")) && !int_in(t, -1, 2, s.rparam)) { err = "bad rparam"; return nullptr; }
        if ((t = sv.get("pscale")) && !int_in(t, 0, 1, s.pscale)) { err = "bad pscale"; return nullptr; }
        g->surf.push_back(s);
    }
    v = doc.get("universes");
    if (!v || v->kind != oj::Val::ARR || v->arr.empty()) { err = "missing universes"; return nullptr; }
    for (auto& uv : v->arr) {
        Universe U;
        const oj::Val* t = uv.get("type");
        if (!t || t->kind != oj::Val::STR) { err = "bad universe"; return nullptr; }
        if (t->str == "csg") {
            U.type = U_CSG;
            const oj::Val* cs = uv.get("cells");
            if (!cs || cs->kind != oj::Val::ARR) { err = "csg universe without cells"; return nullptr; }
            for (auto& cv : cs->arr) {
                Cell c;
                const oj::Val* ss = cv.get("surfaces");
                if (!ss || ss->kind != oj::Val::ARR) { err = "cell without surfaces"; return nullptr; }
                for (auto& pr : ss->arr) {
                    int sid, sn;
                    if (pr.kind != oj::Val::ARR || pr.arr.size() != 2 || !int_in(&pr.arr[0], 0, double(g->surf.size()) - 1, sid) ||
                        !int_in(&pr.arr[1], -1, 1, sn) || sn == 0) { err = "bad cell surface"; return nullptr; }
                    c.surf.push_back(sid); c.sense.push_back(sn);
                }
                const oj::Val* m = cv.get("material");
                const oj::Val* f = cv.get("fill");
                if (m && m->kind == oj::Val::NUM) {
                    if (!int_in(m, 0, double(g->sigma.size()) - 1, c.material)) { err = "bad material"; return nullptr; }
                } else if (f && f->kind == oj::Val::NUM) {
                    if (!int_in(f, 0, 2147483647.0, c.daughter)) { err = "bad cell fill"; return nullptr; }
                    std::vector<double> tr;
                    if (nums(cv.get("translation"), tr)) {
                        if (tr.size() != 3 || !finite_all(tr)) { err = "bad translation"; return nullptr; }
                        for (int d = 0; d < 3; ++d) c.tr[d] = tr[d];
                    }
                } else { err = "cell needs material or fill"; return nullptr; }
                U.cells.push_back(c);
            }
        } else if (t->str == "rect") {
            U.type = U_RECT;
            const oj::Val* gr = uv.get("grid");
            if (!gr || gr->kind != oj::Val::ARR || gr->arr.size() != 3) { err = "rect needs 3 grids"; return nullptr; }
            size_t ne = 1;
            for (int d = 0; d < 3; ++d) {
                if (!nums(&gr->arr[d], U.grid[d]) || U.grid[d].size() < 2 || !finite_all(U.grid[d])) { err = "bad grid"; return nullptr; }
                for (size_t i = 1; i < U.grid[d].size(); ++i)
                    if (!(U.grid[d][i] > U.grid[d][i - 1])) { err = "grid not increasing"; return nullptr; }
                ne *= U.grid[d].size() - 1;
            }
            std::vector<double> fl;
            if (!nums(uv.get("fill"), fl) || fl.size() != ne) { err = "bad rect fill"; return nullptr; }
            for (double x : fl) {
                if (!(x >= 0.0 && x < 2147483647.0) || x != std::floor(x)) { err = "bad lattice fill"; return nullptr; }
                U.fill.push_back(int(x));
            }
            const oj::Val* b = uv.get("bc");
            if (b && b->kind == oj::Val::ARR && b->arr.size() == 6)
                for (int i = 0; i < 6; ++i) U.bc[i] = parse_bc(&b->arr[i]);
            if ((t = uv.get("pscale")) && !int_in(t, 0, 1, U.pscale)) { err = "bad pscale"; return nullptr; }
        } else if (t->str == "hex") {
            U.type = U_HEX;
            const oj::Val* r = uv.get("rings");
            std::vector<double> a1, a2, zz, fl;
            if (!int_in(r, 0, 64, U.rings) || !nums(uv.get("a1"), a1) || !nums(uv.get("a2"), a2) || !nums(uv.get("z"), zz) ||
                a1.size() != 2 || a2.size() != 2 || zz.size() != 2 || !finite_all(a1) || !finite_all(a2) ||
                !finite_all(zz) || !(zz[1] > zz[0]) || !(std::fabs(a1[0] * a2[1] - a2[0] * a1[1]) > 0.0)) {
                err = "bad hex lattice"; return nullptr;
            }
            U.a1[0] = a1[0]; U.a1[1] = a1[1]; U.a2[0] = a2[0]; U.a2[1] = a2[1];
            U.z[0] = zz[0]; U.z[1] = zz[1];
            const oj::Val* nv = uv.get("normals");
            if (!nv || nv->kind != oj::Val::ARR || nv->arr.size() != 3) { err = "hex needs 3 normals"; return nullptr; }
            for (int k = 0; k < 3; ++k) {
                std::vector<double> nk;
                if (!nums(&nv->arr[k], nk) || nk.size() != 2 || !finite_all(nk) || (nk[0] == 0.0 && nk[1] == 0.0)) {
                    err = "bad hex normal"; return nullptr;
                }
                U.nrm[k][0] = nk[0]; U.nrm[k][1] = nk[1];
            }
            const oj::Val* hp = uv.get("half_pitch");
            if (!hp || hp->kind != oj::Val::NUM || !(hp->num > 0.0) || !std::isfinite(hp->num)) { err = "hex needs half_pitch > 0"; return nullptr; }
            U.half_pitch = hp->num;
            for (int rr = -U.rings; rr <= U.rings; ++rr)
                for (int q = std::max(-U.rings, -U.rings - rr); q <= std::min(U.rings, U.rings - rr); ++q) {
                    U.hq.push_back(q); U.hr.push_back(rr);
                }
            if (!nums(uv.get("fill"), fl) || fl.size() != U.hq.size()) { err = "bad hex fill"; return nullptr; }
            for (double x : fl) {
                if (!(x >= 0.0 && x < 2147483647.0) || x != std::floor(x)) { err = "bad lattice fill"; return nullptr; }
                U.fill.push_back(int(x));
            }
            const oj::Val* b = uv.get("bc");
            if (b && b->kind == oj::Val::ARR && b->arr.size() == 3) {
                U.bc[0] = parse_bc(&b->arr[0]); U.bc[4] = parse_bc(&b->arr[1]); U.bc[5] = parse_bc(&b->arr[2]);
            }
        } else { err = "unknown universe type " + t->str; return nullptr; }
        g->univ.push_back(U);
    }
    v = doc.get("root");
    if (!int_in(v, 0, double(g->univ.size()) - 1, g->root)) { err = "missing or bad root"; return nullptr; }
    std::vector<double> sb;
    if (!nums(doc.get("source_box"), sb) || sb.size() != 6 || !finite_all(sb) || !(sb[3] > sb[0]) || !(sb[4] > sb[1]) ||
        !(sb[5] > sb[2])) { err = "missing or empty source_box"; return nullptr; }
    if ((v = doc.get("mesh"))) {
        const oj::Val* mg = v->get("grid");
        if (!mg || mg->kind != oj::Val::ARR || mg->arr.size() != 3) { err = "mesh needs 3 grids"; return nullptr; }
        for (int d = 0; d < 3; ++d) {
            if (!nums(&mg->arr[size_t(d)], g->mesh.grid[d]) || g->mesh.grid[d].size() < 2 || !finite_all(g->mesh.grid[d])) {
                err = "bad mesh grid"; return nullptr;
            }
            for (size_t i = 1; i < g->mesh.grid[d].size(); ++i)
                if (!(g->mesh.grid[d][i] > g->mesh.grid[d][i - 1])) { err = "mesh grid not increasing"; return nullptr; }
        }
    }
    for (int i = 0; i < 6; ++i) g->src[i] = sb[i];
    // references
    for (auto& U : g->univ) {
        for (auto& c : U.cells) {
            if (c.daughter >= int(g->univ.size()) || c.material >= int(g->sigma.size()) ||
                (c.material < 0 && c.daughter < 0)) { err = "bad cell fill"; return nullptr; }
        }
        for (int f : U.fill) if (f < 0 || f >= int(g->univ.size())) { err = "bad lattice fill"; return nullptr; }
    }
    if (count_instances(*g, g->root, 0, err) < 0) return nullptr;
    for (size_t u = 0; u < g->univ.size(); ++u)
        if (g->univ[u].ninst < 0) { err = "universe " + std::to_string(u) + " is not reachable from the root"; return nullptr; }
    g->max_depth = depth_of(*g, g->root);
    // CSG mode: every array as its pseudo-array.  Rect mode: rect arrays by
    // index (Alg. 5/6/9/10); hex arrays, for which the paper gives no array
    // tracker, as their pseudo-arrays (the array tracker's closed-form hex
    // search must return the cell this scan returns).
    for (int u = 0; u < int(g->univ.size()); ++u) {
        const int t = g->univ[u].type;
        if (t == U_CSG) continue;
        if (mode == 1 || t == U_HEX) to_pseudo_array(*g, u, u == g->root);
    }
    return g.release();
}

// ---------------------------------------------------------------------------
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// Round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2;
//        c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0);  key += (W0, W1) between rounds.
// ---------------------------------------------------------------------------
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = uint64_t(M0) * c[0];
        uint64_t p1 = uint64_t(M1) * c[2];
        uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
        uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Reading (counter layout): key = (seed_lo32, geometry_id), counter =
// (particle id, event, tag, k).  Two uniform doubles in (0, 1] per call:
// xi = ((u64 >> 11) + 1) * 2^-53 with u64 = (o1<<32)|o0 and (o3<<32)|o2.
enum { TAG_POSITION = 0, TAG_DIRECTION = 1, TAG_SCALARS = 2, TAG_FISSION = 3, TAG_BANK = 4 };
static void uniform2(uint32_t pid, uint32_t event, uint32_t tag, uint32_t k, uint32_t seed_lo,
                     uint32_t gid, double out[2]) {
    uint32_t ctr[4] = {pid, event, tag, k}, key[2] = {seed_lo, gid}, o[4];
    philox4x32_10(ctr, key, o);
    uint64_t a = (uint64_t(o[1]) << 32) | o[0];
    uint64_t b = (uint64_t(o[3]) << 32) | o[2];
    out[0] = double((a >> 11) + 1) * 0x1.0p-53;
    out[1] = double((b >> 11) + 1) * 0x1.0p-53;
}

// Natural log from + - * / only (so that it is reproducible on any IEEE
// machine): x = 2^k * m with m in [sqrt(1/2), sqrt(2)),
// log m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (m-1)/(m+1),
// |s| <= 0.1716, summed through s^27 by Horner in z = s^2;
// log x = k*LN2_HI + (log m + k*LN2_LO), LN2_HI = ln 2 rounded to 32
// significant bits (so k*LN2_HI is exact), LN2_LO = ln 2 - LN2_HI.
static const double LN2_HI = 0x1.62e42fefp-1;
static const double LN2_LO = 0x1.473de6af278edp-34;
static Real own_log(Real x) {
    uint64_t bits;
    double xd = dv(x);
    std::memcpy(&bits, &xd, 8);
    int k = int((bits >> 52) & 0x7ff) - 1023;
    uint64_t mb = (bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double md;
    std::memcpy(&md, &mb, 8);
    Real m = md;
    if (m > Real(1.4142135623730951)) { m = m * 0.5; k += 1; }
    Real s = (m - 1.0) / (m + 1.0);
    Real z = s * s;
    Real p = 1.0 / 27.0;
    const double coef[13] = {1.0 / 25.0, 1.0 / 23.0, 1.0 / 21.0, 1.0 / 19.0, 1.0 / 17.0, 1.0 / 15.0,
                             1.0 / 13.0, 1.0 / 11.0, 1.0 / 9.0, 1.0 / 7.0, 1.0 / 5.0, 1.0 / 3.0, 1.0};
    for (int i = 0; i < 13; ++i) p = p * z + coef[i];
    Real logm = (s + s) * p;
    Real kd = double(k);
    return kd * LN2_HI + (logm + kd * LN2_LO);
}

// Marsaglia (1972) isotropic direction: u,v uniform on (-1,1], accept
// 0 < s = u^2+v^2 < 1, Omega = (u f, v f, 1 - 2 s) with f = 2 sqrt(1 - s).
// Reading: attempt k uses counter (pid, event, TAG_DIRECTION, k); cap 64.
static bool isotropic(uint32_t pid, uint32_t event, uint32_t seed_lo, uint32_t gid, Real dir[3]) {
    for (uint32_t k = 0; k < 64; ++k) {
        double xi[2];
        uniform2(pid, event, TAG_DIRECTION, k, seed_lo, gid, xi);
        Real u = Real(2.0) * xi[0] - 1.0;
        Real v = Real(2.0) * xi[1] - 1.0;
        Real s = u * u + v * v;
        if (s > Real(0.0) && s < Real(1.0)) {
            Real f = Real(2.0) * rsqrt_(Real(1.0) - s);
            dir[0] = u * f; dir[1] = v * f; dir[2] = Real(1.0) - Real(2.0) * s;
            return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Tracking state: one entry per universe level (level 0 = root).
// ---------------------------------------------------------------------------
static const int MAXL = 8;
struct Level {
    int u = -1;          // universe at this level
    int cell = -1;       // CSG cell index, or array element index
    int ijk[3] = {0, 0, 0};
    Real tr[3];          // translation into the next level's frame
    long long off = 0;   // instance offset contributed by this level
};
struct Particle {
    Real r[3], dir[3], inv[3];
    Real tau = 0.0;
    int nlev = 0;
    Level lv[MAXL];
    int on_lev = -1, on_surf = -1;   // logical "on surface" state
    int material = -1;
    long long inst() const { long long s = 0; for (int l = 0; l < nlev; ++l) s += lv[l].off; return s; }
};

static void set_direction_inverse(Particle& p) {
    for (int d = 0; d < 3; ++d) p.inv[d] = Real(1.0) / p.dir[d];
}

// Reading (frames): the position at level l is the global position minus the
// translations of levels 0..l-1, component by component in level order,
// recomputed from the global position whenever it is needed.
static void local_pos(const Particle& p, int l, Real out[3]) {
    for (int d = 0; d < 3; ++d) out[d] = p.r[d];
    for (int k = 0; k < l; ++k)
        for (int d = 0; d < 3; ++d) out[d] = out[d] - p.lv[k].tr[d];
}

// Reading (sense): f >= 0 is the "+" side.
//   px: f = x - g;  p: f = ((nx x + ny y) + nz z) - d;
//   cz: f = (qx qx + qy qy) - r r with q = (x - x0, y - y0).
static Real surface_f(const Surface& s, const Real x[3]) {
    switch (s.type) {
        case S_PX: return x[0] - s.c[0];
        case S_PY: return x[1] - s.c[0];
        case S_PZ: return x[2] - s.c[0];
        case S_P: return ((Real(s.c[0]) * x[0] + Real(s.c[1]) * x[1]) + Real(s.c[2]) * x[2]) - s.c[3];
        default: {
            Real qx = x[0] - s.c[0], qy = x[1] - s.c[1];
            return (qx * qx + qy * qy) - Real(s.c[2]) * s.c[2];
        }
    }
}
static int sense_at(const Surface& s, const Real x[3]) { return surface_f(s, x) >= Real(0.0) ? +1 : -1; }

// Distance from x along dir to surface s, leaving the side `side` (+1/-1) of
// it; `on` marks the logical on-surface state.  Returns INF for no hit.
// Reading:
//  planes: only the face the direction leaves through is a candidate;
//    px: t = (g - x) * inv_u; p: t = (d - ((nx x + ny y) + nz z)) /
//    ((nx u + ny v) + nz w); a plane the particle is on is never hit again.
//  cz: a = u u + v v, b = qx u + qy v; on the surface and logically inside:
//    t = -2 b / a if b < 0, else no hit; on it and outside: no hit;
//    otherwise c = f, disc = b b - a c, no hit if a == 0 or disc <= 0;
//    inside: t = b <= 0 ? (-b + sqrt disc) / a : -c / (b + sqrt disc);
//    outside: hit only if b < 0, t = c / (-b + sqrt disc).
//  Negative t (the point lies a rounding error outside the cell) becomes 0.
static Real surface_distance(const Surface& s, int side, bool on, const Real x[3], const Real dir[3],
                             const Real inv[3]) {
    Real t = INF;
    switch (s.type) {
        case S_PX: case S_PY: case S_PZ: {
            int d = s.type;
            if (on) return INF;
            bool leaves = side > 0 ? (dir[d] < Real(0.0)) : (dir[d] > Real(0.0));
            if (!leaves) return INF;
            t = (Real(s.c[0]) - x[d]) * inv[d];
            break;
        }
        case S_P: {
            if (on) return INF;
            Real den = (Real(s.c[0]) * dir[0] + Real(s.c[1]) * dir[1]) + Real(s.c[2]) * dir[2];
            bool leaves = side > 0 ? (den < Real(0.0)) : (den > Real(0.0));
            if (!leaves) return INF;
            Real num = Real(s.c[3]) - ((Real(s.c[0]) * x[0] + Real(s.c[1]) * x[1]) + Real(s.c[2]) * x[2]);
            t = num / den;
            break;
        }
        default: {
            Real qx = x[0] - s.c[0], qy = x[1] - s.c[1];
            Real a = dir[0] * dir[0] + dir[1] * dir[1];
            Real b = qx * dir[0] + qy * dir[1];
            if (on) {
                if (side < 0 && b < Real(0.0)) t = (Real(-2.0) * b) / a;
                else return INF;
                break;
            }
            Real c = (qx * qx + qy * qy) - Real(s.c[2]) * s.c[2];
            if (a == Real(0.0)) return INF;
            Real disc = b * b - a * c;
            if (disc <= Real(0.0)) return INF;
            Real sq = rsqrt_(disc);
            if (side < 0) {
                if (b <= Real(0.0)) t = (-b + sq) / a;
                else t = -c / (b + sq);
            } else {
                if (!(b < Real(0.0))) return INF;
                t = c / (-b + sq);
            }
        }
    }
    if (t < Real(0.0)) t = 0.0;
    return t;
}

static bool cell_contains(const Geometry& g, const Cell& c, const Real x[3]) {
    for (size_t i = 0; i < c.surf.size(); ++i)
        if (sense_at(g.surf[c.surf[i]], x) != c.sense[i]) return false;
    return true;
}

// Alg. 5: index of the rect element holding x in one dimension.
// Reading: element i holds g_i <= x < g_{i+1}; a root array has nothing
// outside [g_0, g_n); a non-root array clamps to its border elements (their
// outer faces belong to the parent level).
static int rect_index(const std::vector<double>& gr, Real x, bool is_root) {
    int n = int(gr.size()) - 1;
    if (is_root && (!(Real(gr[0]) <= x) || !(x < Real(gr[n])))) return -1;
    int lo = 0, hi = n - 1;  // answer in [lo, hi]: count of interior planes <= x
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (Real(gr[mid]) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

static void enter_cell(const Geometry& g, Particle& p, int l, int cell) {
    Level& L = p.lv[l];
    const Universe& U = g.univ[L.u];
    const Cell& c = U.cells[cell];
    L.cell = cell;
    L.off = c.off;
    for (int d = 0; d < 3; ++d) L.tr[d] = c.tr[d];
}

static void enter_element(const Geometry& g, Particle& p, int l, const int ijk[3]) {
    Level& L = p.lv[l];
    const Universe& U = g.univ[L.u];
    int n0 = int(U.grid[0].size()) - 1, n1 = int(U.grid[1].size()) - 1;
    int e = ijk[0] + n0 * (ijk[1] + n1 * ijk[2]);
    for (int d = 0; d < 3; ++d) L.ijk[d] = ijk[d];
    L.cell = e;
    L.off = U.eoff[e];
    double t[3];
    rect_center(U, ijk[0], ijk[1], ijk[2], t);
    for (int d = 0; d < 3; ++d) L.tr[d] = t[d];
}

// Daughter universe of the cell/element held at level l (-1 for a material cell).
static int daughter_of(const Geometry& g, const Particle& p, int l) {
    const Universe& U = g.univ[p.lv[l].u];
    if (U.type == U_CSG) return U.cells[p.lv[l].cell].daughter;
    return U.fill[p.lv[l].cell];
}

// Alg. 7 from level l downward: find the cell at each level and descend into
// daughters until a material cell.  Returns false if no cell holds the point.
static bool find_cell_from(const Geometry& g, Particle& p, int l) {
    Real x[3];
    local_pos(p, l, x);
    for (;;) {
        if (l >= MAXL) return false;
        Level& L = p.lv[l];
        const Universe& U = g.univ[L.u];
        bool is_root = (l == 0);
        if (U.type == U_CSG) {
            int found = -1;
            for (size_t c = 0; c < U.cells.size(); ++c)       // Alg. 3: linear scan
                if (cell_contains(g, U.cells[c], x)) { found = int(c); break; }
            if (found < 0) return false;
            enter_cell(g, p, l, found);
        } else {
            int ijk[3];
            for (int d = 0; d < 3; ++d) {
                ijk[d] = rect_index(U.grid[d], x[d], is_root);
                if (ijk[d] < 0) return false;
            }
            enter_element(g, p, l, ijk);
        }
        int dau = daughter_of(g, p, l);
        if (dau < 0) {
            p.nlev = l + 1;
            p.material = U.cells[p.lv[l].cell].material;
            return true;
        }
        for (int d = 0; d < 3; ++d) x[d] = x[d] - L.tr[d];
        p.lv[l + 1].u = dau;
        ++l;
    }
}

// Root-level containment (source rejection): is x inside some root cell?
static bool inside_root(const Geometry& g, const Real x[3]) {
    const Universe& U = g.univ[g.root];
    if (U.type == U_CSG) {
        for (auto& c : U.cells) if (cell_contains(g, c, x)) return true;
        return false;
    }
    for (int d = 0; d < 3; ++d) if (rect_index(U.grid[d], x[d], true) < 0) return false;
    return true;
}

// distance_to_surface over all levels (Table 1).  Reading: levels are scanned
// top to bottom and, within a level, candidates in a fixed order (rect: x, y,
// z; CSG: the cell's surface order) with a strict '<', so that on a tie the
// top-most level wins (the particle crosses at the least embedded level,
// Sec. 3.2).  Rect candidates: the face the direction leaves through in each
// dimension, t = (g - x) * inv; a non-root array has no outer faces.
struct Hit { Real d; int level; int surf; int dim; int dsign; };
static Hit distance_to_boundary(const Geometry& g, const Particle& p) {
    Hit h{INF, -1, -1, -1, 0};
    Real x[3];
    for (int d = 0; d < 3; ++d) x[d] = p.r[d];
    for (int l = 0; l < p.nlev; ++l) {
        if (l > 0) for (int d = 0; d < 3; ++d) x[d] = x[d] - p.lv[l - 1].tr[d];
        const Level& L = p.lv[l];
        const Universe& U = g.univ[L.u];
        if (U.type == U_CSG) {
            const Cell& c = U.cells[L.cell];
            for (size_t i = 0; i < c.surf.size(); ++i) {
                bool on = (p.on_lev == l && p.on_surf == c.surf[i]);
                Real t = surface_distance(g.surf[c.surf[i]], c.sense[i], on, x, p.dir, p.inv);
                if (t < h.d) { h.d = t; h.level = l; h.surf = c.surf[i]; h.dim = -1; }
            }
        } else {
            for (int d = 0; d < 3; ++d) {
                int n = int(U.grid[d].size()) - 1;
                int i = L.ijk[d];
                Real t = INF;
                int sg = 0;
                if (p.dir[d] > Real(0.0)) {
                    if (i < n - 1 || l == 0) { t = (Real(U.grid[d][i + 1]) - x[d]) * p.inv[d]; sg = +1; }
                } else if (p.dir[d] < Real(0.0)) {
                    if (i > 0 || l == 0) { t = (Real(U.grid[d][i]) - x[d]) * p.inv[d]; sg = -1; }
                }
                if (sg != 0 && t < Real(0.0)) t = 0.0;
                if (sg != 0 && t < h.d) { h.d = t; h.level = l; h.surf = -1 - (2 * d + (sg > 0)); h.dim = d; h.dsign = sg; }
            }
        }
    }
    return h;
}

enum CrossResult { CR_OK = 0, CR_REFLECT = 1, CR_ESCAPE = 2, CR_LOST = 3 };

// Reflection off a root plane: axis planes negate one component; a general
// plane maps dir -> dir - k n, k = 2 (n.dir) / (n.n).
static void reflect(Particle& p, const Surface* s, int dim) {
    if (s == nullptr || s->type <= S_PZ) {
        int d = s ? s->type : dim;
        p.dir[d] = -p.dir[d];
    } else {
        Real nd = (Real(s->c[0]) * p.dir[0] + Real(s->c[1]) * p.dir[1]) + Real(s->c[2]) * p.dir[2];
        Real nn = (Real(s->c[0]) * s->c[0] + Real(s->c[1]) * s->c[1]) + Real(s->c[2]) * s->c[2];
        Real k = (Real(2.0) * nd) / nn;
        for (int d = 0; d < 3; ++d) p.dir[d] = p.dir[d] - k * s->c[d];
    }
    set_direction_inverse(p);
}

// Alg. 8 (with Alg. 4 / Alg. 6 at the crossing level).
static int cross_surface(const Geometry& g, Particle& p, const Hit& h) {
    int l = h.level;
    Level& L = p.lv[l];
    const Universe& U = g.univ[L.u];
    if (U.type == U_CSG) {
        Real x[3];
        local_pos(p, l, x);
        const Cell& old = U.cells[L.cell];
        int old_sense = 0;
        for (size_t i = 0; i < old.surf.size(); ++i) if (old.surf[i] == h.surf) old_sense = old.sense[i];
        int found = -1;
        for (size_t ci = 0; ci < U.cells.size() && found < 0; ++ci) {   // Alg. 4
            if (int(ci) == L.cell) continue;
            const Cell& c = U.cells[ci];
            bool ok = true;
            for (size_t i = 0; i < c.surf.size() && ok; ++i) {
                if (c.surf[i] == h.surf) ok = (c.sense[i] == -old_sense);   // logical flip
                else ok = (sense_at(g.surf[c.surf[i]], x) == c.sense[i]);
            }
            if (ok) found = int(ci);
        }
        p.on_lev = l;
        p.on_surf = h.surf;
        if (found < 0) {
            if (l != 0) return CR_LOST;
            const Surface& s = g.surf[h.surf];
            if (s.bc == BC_REFLECT) { reflect(p, &s, -1); return CR_REFLECT; }
            return CR_ESCAPE;
        }
        enter_cell(g, p, l, found);
    } else {
        int ijk[3] = {L.ijk[0], L.ijk[1], L.ijk[2]};             // Alg. 6
        ijk[h.dim] += h.dsign;
        int n = int(U.grid[h.dim].size()) - 1;
        p.on_lev = l;
        p.on_surf = h.surf;
        if (ijk[h.dim] < 0 || ijk[h.dim] >= n) {
            if (l != 0) return CR_LOST;
            int bc = U.bc[2 * h.dim + (h.dsign > 0)];
            if (bc == BC_REFLECT) { reflect(p, nullptr, h.dim); return CR_REFLECT; }
            return CR_ESCAPE;
        }
        enter_element(g, p, l, ijk);
    }
    int dau = daughter_of(g, p, l);
    if (dau < 0) {
        p.nlev = l + 1;
        p.material = U.cells[p.lv[l].cell].material;
        return CR_OK;
    }
    p.lv[l + 1].u = dau;
    return find_cell_from(g, p, l + 1) ? CR_OK : CR_LOST;
}

// ---------------------------------------------------------------------------
// Birth (Alg. 2, lines "sample position/direction"), Reading:
// position lo + xi (hi - lo) over the source box, attempt a uses counters
// (pid, 0, TAG_POSITION, 2a) -> (xi_x, xi_y) and (pid, 0, TAG_POSITION, 2a+1)
// -> xi_z; points outside every root cell are rejected (cap 1e6 attempts);
// direction isotropic at event 0; tau = -log(xi) with xi the second number of
// counter (pid, 0, TAG_SCALARS, 0).
// ---------------------------------------------------------------------------
enum PStatus { P_ALIVE = 0, P_ABSORBED = 1, P_ESCAPED = 2, P_CUTOFF = 3,
               P_LOST = -5, P_MAXSEG = -6, P_SOURCE = -9 };

static int sample_birth(const Geometry& g, uint32_t pid, uint32_t seed_lo, Real r[3], Real dir[3], Real& tau) {
    uint32_t gid = uint32_t(g.gid);
    bool placed = false;
    for (uint32_t a = 0; a < 1000000u && !placed; ++a) {
        double xy[2], zz[2];
        uniform2(pid, 0, TAG_POSITION, 2 * a, seed_lo, gid, xy);
        uniform2(pid, 0, TAG_POSITION, 2 * a + 1, seed_lo, gid, zz);
        double xi[3] = {xy[0], xy[1], zz[0]};
        for (int d = 0; d < 3; ++d) r[d] = Real(g.src[d]) + Real(xi[d]) * (Real(g.src[3 + d]) - g.src[d]);
        placed = inside_root(g, r);
    }
    if (!placed) return P_SOURCE;
    if (!isotropic(pid, 0, seed_lo, gid, dir)) return P_SOURCE;
    double sc[2];
    uniform2(pid, 0, TAG_SCALARS, 0, seed_lo, gid, sc);
    tau = -own_log(sc[1]);
    return P_ALIVE;
}

// Counters shared in meaning with the library's device counters.
enum { K_SEGMENTS = 0, K_CROSSINGS, K_COLLISIONS, K_ABSORBED, K_ESCAPED, K_REFLECTIONS, K_LOST,
       K_MAXSEG, K_CUTOFF, K_SOURCE, K_NCOUNTERS = 16 };

// FNV-1a over 64-bit words: a per-particle digest of (instance, segment length bits).
static inline uint64_t fnv(uint64_t h, uint64_t w) { return (h ^ w) * 0x100000001b3ULL; }
static const uint64_t FNV0 = 0xcbf29ce484222325ULL;

struct RunOpts {
    double p_absorb = 0.3;
    long long max_segments = 1000000;
    double max_path = INF;
};

struct HistoryOut {
    int status = 0;
    long long nseg = 0;
    uint64_t hash = FNV0;
    double fin[3] = {0, 0, 0};
    int nsites = 0;                 // fission sites banked at the absorption (power iteration)
    uint64_t nu_fixed = 0;          // llrint(nu * 2^32) of the absorbing material
};

// Power iteration (reading of Alg. 1 with a synthetic fission source): an
// absorption in material m with nu_m > 0 banks floor(nu_m / k + xi) sites at
// the absorption point, at most FISSION_MAX (k: the previous cycle's
// estimate, 1 in the first; xi: first value of counter (pid, e, TAG_FISSION,
// 0), e the absorbing collision's event number) and adds llrint(nu_m * 2^32)
// to the cycle's nu sum.
constexpr int FISSION_MAX = 8;

// Mesh track-length tally of one segment (reading): the segment starts at
// p.r and runs `len` along p.dir.  Per axis, with planes g_0 < ... < g_n,
// the start's index is the largest i in -1..n with g_i <= x (g_-1 = -inf):
// -1 and n are the two sides outside the mesh.  From the start, per axis
// with a nonzero direction component, the next plane is g_{i+1} moving up
// (none from index n) or g_i moving down (none from index -1), at
// t = (g - x0) * (1/u) measured from the segment start.  A piece ends at the
// smallest such t below len (ties: x before y before z; a t equal to len is
// no crossing); a t below the piece's start counts as the start.  A piece
// whose three indices are inside the mesh is tallied as
// llrint(length * 2^32) into its bin (x fastest, then y, then z); the index
// then steps along the crossing axis, until the walk reaches len.
static void mesh_walk(const Geometry& g, const Particle& p, Real len, uint64_t* mesh) {
    const Mesh& M = g.mesh;
    int n[3], idx[3];
    for (int d = 0; d < 3; ++d) {
        const std::vector<double>& gr = M.grid[d];
        n[d] = int(gr.size()) - 1;
        const double x = dv(p.r[d]);
        int i = -1;
        while (i + 1 <= n[d] && gr[size_t(i + 1)] <= x) ++i;
        idx[d] = i;
    }
    Real t0 = 0.0;
    for (;;) {
        Real tn = len;
        int ax = -1;
        for (int d = 0; d < 3; ++d) {
            Real t;
            if (p.dir[d] > Real(0.0) && idx[d] < n[d]) t = (Real(M.grid[d][size_t(idx[d] + 1)]) - p.r[d]) * p.inv[d];
            else if (p.dir[d] < Real(0.0) && idx[d] >= 0) t = (Real(M.grid[d][size_t(idx[d])]) - p.r[d]) * p.inv[d];
            else continue;
            if (t < tn) { tn = t; ax = d; }
        }
        if (tn < t0) tn = t0;
        if (idx[0] >= 0 && idx[0] < n[0] && idx[1] >= 0 && idx[1] < n[1] && idx[2] >= 0 && idx[2] < n[2]) {
            const long long b = idx[0] + (long long)n[0] * (idx[1] + (long long)n[1] * idx[2]);
            mesh[b] += uint64_t(std::llrint(dv((tn - t0) * 4294967296.0)));
        }
        if (ax < 0) break;
        t0 = tn;
        idx[ax] += p.dir[ax] > Real(0.0) ? 1 : -1;
    }
}

// One history of Alg. 2 with the synthetic physics.  Reading (flight):
//   dc = tau / Sigma (Sigma = 0 -> +inf);
//   if d < dc: tally(d); r = r + d*Omega; tau = tau - Sigma*d; cross;
//   else:      tally(dc); r = r + dc*Omega; collide;
// tally adds llrint(len * 2^32) to the leaf instance's 64-bit bin.
// Collision e (1-based): (xi_abs, xi_tau) from counter (pid, e, TAG_SCALARS,
// 0); absorbed iff xi_abs < p_a; else new isotropic direction at event e and
// tau = -log(xi_tau); the on-surface state is cleared.
// A path cutoff (test-only option) ends the history once the accumulated
// track length reaches max_path, tallying only the part up to it.
// Birth from a fission bank of B sites (xyz triples, B > 0): site
// floor(xi * B) (xi: first value of counter (pid, 0, TAG_BANK, 0), B - 1 at
// xi = 1), direction and tau as from the source box.
static int sample_birth_bank(const Geometry& g, uint32_t pid, uint32_t seed_lo, const std::vector<double>& bank,
                             Real r[3], Real dir[3], Real& tau) {
    const uint32_t gid = uint32_t(g.gid);
    const long long B = (long long)(bank.size() / 3);
    double xb[2];
    uniform2(pid, 0, TAG_BANK, 0, seed_lo, gid, xb);
    long long j = (long long)std::floor(xb[0] * double(B));
    if (j >= B) j = B - 1;
    for (int d = 0; d < 3; ++d) r[d] = bank[size_t(3 * j + d)];
    if (!isotropic(pid, 0, seed_lo, gid, dir)) return P_SOURCE;
    double sc[2];
    uniform2(pid, 0, TAG_SCALARS, 0, seed_lo, gid, sc);
    tau = -own_log(sc[1]);
    return P_ALIVE;
}

template <class Trace>
static HistoryOut run_one(const Geometry& g, uint32_t pid, uint32_t seed_lo, const RunOpts& o,
                          uint64_t* tally, unsigned long long* cnt, Trace&& trace, uint64_t* mesh = nullptr,
                          const std::vector<double>* bank = nullptr, double knorm = 0.0) {
    HistoryOut out;
    Particle p;
    Real tau;
    out.status = bank ? sample_birth_bank(g, pid, seed_lo, *bank, p.r, p.dir, tau)
                      : sample_birth(g, pid, seed_lo, p.r, p.dir, tau);
    if (out.status != P_ALIVE) { cnt[K_SOURCE]++; return out; }
    p.tau = tau;
    set_direction_inverse(p);
    p.lv[0].u = g.root;
    if (!find_cell_from(g, p, 0)) { out.status = P_LOST; cnt[K_LOST]++; return out; }
    uint32_t event = 0;
    Real path = 0.0;
    bool cutoff = std::isfinite(o.max_path);
    for (;;) {
        Hit h = distance_to_boundary(g, p);
        Real sig = g.sigma[p.material];
        Real dc = sig > Real(0.0) ? p.tau / sig : Real(INF);
        bool crossing = h.d < dc;
        Real len = crossing ? h.d : dc;
        if (!(len < Real(INF))) { out.status = P_LOST; cnt[K_LOST]++; break; }
        long long inst = p.inst();
        bool stop_cut = false;
        if (cutoff && path + len >= Real(o.max_path)) { len = Real(o.max_path) - path; stop_cut = true; }
        else path = path + len;
        long long q = std::llrint(dv(len * 4294967296.0));
        tally[inst] += uint64_t(q);
        if (mesh) mesh_walk(g, p, len, mesh);
        uint64_t lb;
        double ld = dv(len);
        std::memcpy(&lb, &ld, 8);
        out.hash = fnv(fnv(out.hash, uint64_t(inst)), lb);
        trace(inst, ld, crossing ? (stop_cut ? 2 : 0) : (stop_cut ? 2 : 1), p);
        for (int d = 0; d < 3; ++d) p.r[d] = p.r[d] + len * p.dir[d];
        out.nseg++;
        cnt[K_SEGMENTS]++;
        if (stop_cut) { out.status = P_CUTOFF; cnt[K_CUTOFF]++; break; }
        if (crossing) {
            p.tau = p.tau - sig * h.d;
            cnt[K_CROSSINGS]++;
            int cr = cross_surface(g, p, h);
            if (cr == CR_ESCAPE) { out.status = P_ESCAPED; cnt[K_ESCAPED]++; break; }
            if (cr == CR_LOST) { out.status = P_LOST; cnt[K_LOST]++; break; }
            if (cr == CR_REFLECT) cnt[K_REFLECTIONS]++;
        } else {
            ++event;
            cnt[K_COLLISIONS]++;
            double sc[2];
            uniform2(pid, event, TAG_SCALARS, 0, seed_lo, uint32_t(g.gid), sc);
            if (sc[0] < o.p_absorb) {
                out.status = P_ABSORBED;
                cnt[K_ABSORBED]++;
                const double nu = g.nu[size_t(p.material)];
                if (knorm > 0.0 && nu > 0.0) {
                    double xf[2];
                    uniform2(pid, event, TAG_FISSION, 0, seed_lo, uint32_t(g.gid), xf);
                    const double ns = std::floor(nu / knorm + xf[0]);
                    out.nsites = ns > double(FISSION_MAX) ? FISSION_MAX : int(ns);
                    out.nu_fixed = uint64_t(std::llrint(nu * 4294967296.0));
                }
                break;
            }
            if (!isotropic(pid, event, seed_lo, uint32_t(g.gid), p.dir)) { out.status = P_LOST; cnt[K_LOST]++; break; }
            set_direction_inverse(p);
            p.tau = -own_log(sc[1]);
            p.on_lev = -1; p.on_surf = -1;
        }
        if (out.nseg >= o.max_segments) { out.status = P_MAXSEG; cnt[K_MAXSEG]++; break; }
    }
    for (int d = 0; d < 3; ++d) out.fin[d] = dv(p.r[d]);
    return out;
}

// ---------------------------------------------------------------------------
// Brute-force find_cell over every leaf instance in the global frame (the
// pin for the hierarchical walk): each leaf instance is the intersection of
// all constraints along its chain of cells, each constraint evaluated on a
// surface moved into the global frame.
// ---------------------------------------------------------------------------
struct GConstraint { int type; double c[4]; int sense; };   // global-frame surface
struct GLeaf { std::vector<GConstraint> cons; };

static void enumerate_leaves(const Geometry& g, int u, const double T[3], std::vector<GConstraint>& chain,
                             bool is_root, std::vector<GLeaf>& out) {
    const Universe& U = g.univ[u];
    auto moved = [&](const Surface& s, int sense) {
        GConstraint k; k.type = s.type; k.sense = sense;
        for (int i = 0; i < 4; ++i) k.c[i] = s.c[i];
        if (s.type <= S_PZ) k.c[0] = s.c[0] + T[s.type];
        else if (s.type == S_P) k.c[3] = s.c[3] + (s.c[0] * T[0] + s.c[1] * T[1] + s.c[2] * T[2]);
        else { k.c[0] = s.c[0] + T[0]; k.c[1] = s.c[1] + T[1]; }
        return k;
    };
    if (U.type == U_CSG) {
        for (auto& c : U.cells) {
            size_t base = chain.size();
            for (size_t i = 0; i < c.surf.size(); ++i) chain.push_back(moved(g.surf[c.surf[i]], c.sense[i]));
            if (c.material >= 0) out.push_back(GLeaf{chain});
            else {
                double T2[3] = {T[0] + c.tr[0], T[1] + c.tr[1], T[2] + c.tr[2]};
                enumerate_leaves(g, c.daughter, T2, chain, false, out);
            }
            chain.resize(base);
        }
        return;
    }
    int n[3] = {int(U.grid[0].size()) - 1, int(U.grid[1].size()) - 1, int(U.grid[2].size()) - 1};
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                size_t base = chain.size();
                int ijk[3] = {i, j, k};
                for (int d = 0; d < 3; ++d) {
                    if (ijk[d] > 0 || is_root) { GConstraint c{d, {U.grid[d][ijk[d]] + T[d], 0, 0, 0}, +1}; chain.push_back(c); }
                    if (ijk[d] < n[d] - 1 || is_root) { GConstraint c{d, {U.grid[d][ijk[d] + 1] + T[d], 0, 0, 0}, -1}; chain.push_back(c); }
                }
                double t[3];
                rect_center(U, i, j, k, t);
                double T2[3] = {T[0] + t[0], T[1] + t[1], T[2] + t[2]};
                enumerate_leaves(g, U.fill[i + n[0] * (j + n[1] * k)], T2, chain, false, out);
                chain.resize(base);
            }
}

static double gc_f(const GConstraint& k, const double x[3], double* grad) {
    switch (k.type) {
        case S_PX: case S_PY: case S_PZ: *grad = 1.0; return x[k.type] - k.c[0];
        case S_P: *grad = std::sqrt(k.c[0] * k.c[0] + k.c[1] * k.c[1] + k.c[2] * k.c[2]);
                  return k.c[0] * x[0] + k.c[1] * x[1] + k.c[2] * x[2] - k.c[3];
        default: {
            double qx = x[0] - k.c[0], qy = x[1] - k.c[1];
            double rr = std::sqrt(qx * qx + qy * qy);
            *grad = 1.0;   // report |r - R| as the distance for cylinders
            return rr - k.c[2];
        }
    }
}

// ---------------------------------------------------------------------------
// Transmission along deterministic rays (no collisions): per-material track
// lengths, T = exp(-sum sigma_m l_m), and the analytic derivative of T with
// respect to sigma_m and to the design parameters theta = (r_0, r_1, r_2,
// pitch).  At a crossing of surface f(x; theta) = 0 the hit distance moves by
// dt/dtheta = -(df/dtheta) / (grad f . Omega); each segment's length moves by
// dt_exit - dt_entry.  Planes and cylinder centres tagged "pscale" sit at
// G = k * pitch in the global frame (dG/dpitch = G / pitch); a cylinder
// tagged rparam = j has df/dr_j = -2 r_j.
// ---------------------------------------------------------------------------
static const int NPARAM = 4;

static void hit_derivative(const Geometry& g, const Particle& p, const Hit& h, double pitch, double out[NPARAM]) {
    for (int j = 0; j < NPARAM; ++j) out[j] = 0.0;
    const Universe& U = g.univ[p.lv[h.level].u];
    double T[3] = {0, 0, 0};                       // translation of level h.level's frame
    for (int k = 0; k < h.level; ++k) for (int d = 0; d < 3; ++d) T[d] += dv(p.lv[k].tr[d]);
    double dir[3] = {dv(p.dir[0]), dv(p.dir[1]), dv(p.dir[2])};
    double x[3] = {dv(p.r[0]), dv(p.r[1]), dv(p.r[2])};
    if (U.type != U_CSG || h.surf < 0) {
        // rect array plane of dimension h.dim
        if (h.dim < 2 && U.pscale && pitch > 0) {
            const std::vector<double>& gr = U.grid[h.dim];
            double G = gr[p.lv[h.level].ijk[h.dim] + (h.dsign > 0)] + T[h.dim];
            out[3] = (G / pitch) / dir[h.dim];
        }
        return;
    }
    const Surface& s = g.surf[h.surf];
    if (s.type <= S_PY) {
        if (s.pscale && pitch > 0) {
            double G = s.c[0] + T[s.type];
            out[3] = (G / pitch) / dir[s.type];
        }
    } else if (s.type == S_CZ) {
        double cx = s.c[0] + T[0], cy = s.c[1] + T[1];
        double qx = x[0] - cx, qy = x[1] - cy;
        double gd = 2.0 * (qx * dir[0] + qy * dir[1]);
        if (gd == 0.0) return;
        if (s.rparam >= 0 && s.rparam < 3) out[s.rparam] = -(-2.0 * s.c[2]) / gd;
        if (s.pscale && pitch > 0) out[3] = -(-2.0 * (qx * cx + qy * cy) / pitch) / gd;
    }
}

static void transmit_one(const Geometry& g, const double ray[6], const double* sigma, double pitch,
                         double& T, double* lens, double* dT, uint64_t& hash, int& status) {
    int nm = int(g.sigma.size());
    std::vector<double> dl(size_t(nm) * NPARAM, 0.0);
    for (int m = 0; m < nm; ++m) lens[m] = 0.0;
    hash = FNV0;
    status = 0;
    Particle p;
    for (int d = 0; d < 3; ++d) { p.r[d] = ray[d]; p.dir[d] = ray[3 + d]; }
    set_direction_inverse(p);
    p.lv[0].u = g.root;
    double dt_in[NPARAM] = {0, 0, 0, 0};
    if (!find_cell_from(g, p, 0)) { status = P_LOST; T = 1.0; goto done; }
    for (long long seg = 0; seg < 10000000; ++seg) {
        Hit h = distance_to_boundary(g, p);
        if (!(h.d < Real(INF))) { status = P_LOST; break; }
        int m = p.material;
        long long inst = p.inst();
        hash = fnv(hash, uint64_t(inst));
        lens[m] += dv(h.d);
        for (int d = 0; d < 3; ++d) p.r[d] = p.r[d] + h.d * p.dir[d];
        double dt_out[NPARAM];
        hit_derivative(g, p, h, pitch, dt_out);
        for (int j = 0; j < NPARAM; ++j) dl[size_t(m) * NPARAM + j] += dt_out[j] - dt_in[j];
        for (int j = 0; j < NPARAM; ++j) dt_in[j] = dt_out[j];
        int cr = cross_surface(g, p, h);
        if (cr == CR_ESCAPE) { status = P_ESCAPED; break; }
        if (cr == CR_LOST) { status = P_LOST; break; }
    }
    {
        double opt = 0.0;
        for (int m = 0; m < nm; ++m) opt += sigma[m] * lens[m];
        T = std::exp(-opt);
    }
done:
    if (dT) {
        for (int m = 0; m < nm; ++m) dT[m] = -lens[m] * T;
        for (int j = 0; j < NPARAM; ++j) {
            double acc = 0.0;
            for (int m = 0; m < nm; ++m) acc += sigma[m] * dl[size_t(m) * NPARAM + j];
            dT[nm + j] = -T * acc;
        }
    }
}

// ---------------------------------------------------------------------------
// C interface (ctypes).
// ---------------------------------------------------------------------------
extern "C" {

void* orc_geometry_load(const char* json, long long len, int mode, char* err, int errlen) {
    std::string e;
    Geometry* g = load_geometry(json, size_t(len), mode, e);
    if (!g && err && errlen > 0) { std::snprintf(err, size_t(errlen), "%s", e.c_str()); }
    return g;
}

void orc_geometry_free(void* g) { delete static_cast<Geometry*>(g); }

long long orc_n_instances(void* gp) {
    Geometry* g = static_cast<Geometry*>(gp);
    return g->univ[g->root].ninst;
}
int orc_n_materials(void* gp) { return int(static_cast<Geometry*>(gp)->sigma.size()); }
int orc_max_depth(void* gp) { return static_cast<Geometry*>(gp)->max_depth; }

// Birth states: out[7*i..] = x y z u v w tau, status[i].
int orc_source(void* gp, long long n, long long first_id, unsigned long long seed, double* out, int* status) {
    Geometry* g = static_cast<Geometry*>(gp);
    for (long long i = 0; i < n; ++i) {
        Real r[3], dir[3], tau = 0.0;
        int st = sample_birth(*g, uint32_t(first_id + i), uint32_t(seed), r, dir, tau);
        for (int d = 0; d < 3; ++d) { out[7 * i + d] = dv(r[d]); out[7 * i + 3 + d] = dv(dir[d]); }
        out[7 * i + 6] = dv(tau);
        if (status) status[i] = st;
    }
    return 0;
}

int orc_run(void* gp, long long n, long long first_id, unsigned long long seed, double p_absorb,
            long long max_segments, double max_path, int nthreads, unsigned long long* tally,
            unsigned long long* counters, unsigned long long* rec_hash, long long* rec_nseg,
            int* rec_status, double* rec_final) {
    Geometry* g = static_cast<Geometry*>(gp);
    RunOpts o;
    o.p_absorb = p_absorb;
    o.max_segments = max_segments;
    o.max_path = max_path;
    long long ninst = g->univ[g->root].ninst;
    if (nthreads < 1) nthreads = 1;
    if (n < nthreads) nthreads = int(std::max<long long>(1, n));
    std::vector<std::vector<uint64_t>> tl(size_t(nthreads), std::vector<uint64_t>(size_t(ninst), 0));
    std::vector<std::vector<unsigned long long>> cl(size_t(nthreads), std::vector<unsigned long long>(K_NCOUNTERS, 0));
    auto work = [&](int t) {
        long long lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
        for (long long i = lo; i < hi; ++i) {
            HistoryOut h = run_one(*g, uint32_t(first_id + i), uint32_t(seed), o, tl[size_t(t)].data(),
                                   cl[size_t(t)].data(), [](long long, double, int, const Particle&) {});
            if (rec_hash) rec_hash[i] = h.hash;
            if (rec_nseg) rec_nseg[i] = h.nseg;
            if (rec_status) rec_status[i] = h.status;
            if (rec_final) for (int d = 0; d < 3; ++d) rec_final[3 * i + d] = h.fin[d];
        }
    };
    if (nthreads == 1) work(0);
    else {
        std::vector<std::thread> th;
        for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
        for (auto& x : th) x.join();
    }
    for (long long b = 0; b < ninst; ++b) {
        uint64_t s = 0;
        for (int t = 0; t < nthreads; ++t) s += tl[size_t(t)][size_t(b)];
        tally[b] = s;
    }
    for (int k = 0; k < K_NCOUNTERS; ++k) {
        unsigned long long s = 0;
        for (int t = 0; t < nthreads; ++t) s += cl[size_t(t)][size_t(k)];
        counters[k] = s;
    }
    return 0;
}

// orc_run plus the mesh track-length tally (uint64[bins], x fastest).
int orc_run_mesh(void* gp, long long n, long long first_id, unsigned long long seed, double p_absorb, int nthreads,
                 unsigned long long* tally, unsigned long long* counters, unsigned long long* mesh) {
    Geometry* g = static_cast<Geometry*>(gp);
    if (!g->mesh.on()) return -1;
    RunOpts o;
    o.p_absorb = p_absorb;
    o.max_segments = 1000000;
    o.max_path = INF;
    const long long ninst = g->univ[g->root].ninst, nb = g->mesh.bins();
    if (nthreads < 1) nthreads = 1;
    if (n < nthreads) nthreads = int(std::max<long long>(1, n));
    std::vector<std::vector<uint64_t>> tl(size_t(nthreads), std::vector<uint64_t>(size_t(ninst), 0));
    std::vector<std::vector<uint64_t>> ml(size_t(nthreads), std::vector<uint64_t>(size_t(nb), 0));
    std::vector<std::vector<unsigned long long>> cl(size_t(nthreads), std::vector<unsigned long long>(K_NCOUNTERS, 0));
    auto work = [&](int t) {
        long long lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
        for (long long i = lo; i < hi; ++i)
            run_one(*g, uint32_t(first_id + i), uint32_t(seed), o, tl[size_t(t)].data(), cl[size_t(t)].data(),
                    [](long long, double, int, const Particle&) {}, ml[size_t(t)].data());
    };
    if (nthreads == 1) work(0);
    else {
        std::vector<std::thread> th;
        for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
        for (auto& x : th) x.join();
    }
    for (long long b = 0; b < ninst; ++b) {
        uint64_t s = 0;
        for (int t = 0; t < nthreads; ++t) s += tl[size_t(t)][size_t(b)];
        tally[b] = s;
    }
    for (long long b = 0; b < nb; ++b) {
        uint64_t s = 0;
        for (int t = 0; t < nthreads; ++t) s += ml[size_t(t)][size_t(b)];
        mesh[b] = s;
    }
    for (int k = 0; k < K_NCOUNTERS; ++k) {
        unsigned long long s = 0;
        for (int t = 0; t < nthreads; ++t) s += cl[size_t(t)][size_t(k)];
        counters[k] = s;
    }
    return 0;
}

// Power iteration (Alg. 1): `cycles` cycles of n histories, the first
// `inactive` of them not tallied.  Cycle c's particle ids are
// first_id + c*n .. first_id + c*n + n - 1; cycle 0 is born in the source
// box, cycle c > 0 from cycle c-1's bank (its sites in history order).
// k_c = (double(sum over the cycle's fissile absorptions of
// llrint(nu * 2^32)) * 2^-32) / n.  Writes k_out[c] and bank_out[c] (sites
// banked); returns 0, or -1 when a cycle banks no site.
int orc_power(void* gp, long long n, long long first_id, unsigned long long seed, double p_absorb, int inactive,
              int cycles, int nthreads, double* k_out, long long* bank_out, unsigned long long* tally,
              unsigned long long* counters) {
    Geometry* g = static_cast<Geometry*>(gp);
    RunOpts o;
    o.p_absorb = p_absorb;
    o.max_segments = 1000000;
    o.max_path = INF;
    const long long ninst = g->univ[g->root].ninst;
    if (nthreads < 1) nthreads = 1;
    if (n < nthreads) nthreads = int(std::max<long long>(1, n));
    std::vector<double> bank;
    double knorm = 1.0;
    std::vector<uint64_t> tsum(size_t(ninst), 0);
    std::vector<unsigned long long> csum(K_NCOUNTERS, 0);
    for (int c = 0; c < cycles; ++c) {
        const bool active = c >= inactive;
        std::vector<HistoryOut> hist(static_cast<size_t>(n));
        std::vector<std::vector<uint64_t>> tl(size_t(nthreads), std::vector<uint64_t>(size_t(ninst), 0));
        std::vector<std::vector<unsigned long long>> cl(size_t(nthreads), std::vector<unsigned long long>(K_NCOUNTERS, 0));
        const std::vector<double>* src = c == 0 ? nullptr : &bank;
        auto work = [&](int t) {
            long long lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
            for (long long i = lo; i < hi; ++i)
                hist[size_t(i)] = run_one(*g, uint32_t(first_id + (long long)c * n + i), uint32_t(seed), o,
                                          tl[size_t(t)].data(), cl[size_t(t)].data(), [](long long, double, int, const Particle&) {},
                                          nullptr, src, knorm);
        };
        if (nthreads == 1) work(0);
        else {
            std::vector<std::thread> th;
            for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
            for (auto& x : th) x.join();
        }
        uint64_t nusum = 0;
        std::vector<double> next;
        for (long long i = 0; i < n; ++i) {
            const HistoryOut& h = hist[size_t(i)];
            nusum += h.nu_fixed;
            for (int k = 0; k < h.nsites; ++k)
                for (int d = 0; d < 3; ++d) next.push_back(h.fin[d]);
        }
        const double kc = (double(nusum) * 0x1p-32) / double(n);
        k_out[c] = kc;
        bank_out[c] = (long long)(next.size() / 3);
        if (active) {
            for (int t = 0; t < nthreads; ++t) {
                for (long long b = 0; b < ninst; ++b) tsum[size_t(b)] += tl[size_t(t)][size_t(b)];
                for (int k = 0; k < K_NCOUNTERS; ++k) csum[size_t(k)] += cl[size_t(t)][size_t(k)];
            }
        }
        if (next.empty()) return -1;
        bank.swap(next);
        knorm = kc;
    }
    for (long long b = 0; b < ninst; ++b) tally[b] = tsum[size_t(b)];
    for (int k = 0; k < K_NCOUNTERS; ++k) counters[k] = csum[size_t(k)];
    return 0;
}

// Mesh tally of one segment from (x, y, z) along (u, v, w), length len, with
// the direction's reciprocals computed as the tracker does (a test hook).
int orc_mesh_segment(void* gp, const double* r, const double* dir, double len, unsigned long long* mesh) {
    Geometry* g = static_cast<Geometry*>(gp);
    if (!g->mesh.on()) return -1;
    Particle p;
    for (int d = 0; d < 3; ++d) { p.r[d] = r[d]; p.dir[d] = dir[d]; }
    set_direction_inverse(p);
    mesh_walk(*g, p, len, reinterpret_cast<uint64_t*>(mesh));
    return 0;
}

long long orc_mesh_bins(void* gp) { return static_cast<Geometry*>(gp)->mesh.bins(); }

// Per-segment trace of one history: instance, length, kind (0 cross, 1 collide, 2 cutoff).
// One history's segments: leaf instance, length and kind (0 crossing, 1
// collision, 2 cut) per segment and, when `geo` is given, the segment's start
// position and direction in the global frame and its material's cross
// section (7 doubles per segment).
long long orc_trace(void* gp, long long pid, unsigned long long seed, double p_absorb, long long max_segments,
                    long long cap, long long* inst, double* len, int* kind, int* status, double* geo) {
    Geometry* g = static_cast<Geometry*>(gp);
    RunOpts o;
    o.p_absorb = p_absorb;
    o.max_segments = max_segments;
    std::vector<uint64_t> tally(size_t(g->univ[g->root].ninst), 0);
    unsigned long long cnt[K_NCOUNTERS] = {0};
    long long k = 0;
    HistoryOut h = run_one(*g, uint32_t(pid), uint32_t(seed), o, tally.data(), cnt,
                           [&](long long i, double l, int kd, const Particle& p) {
                               if (k < cap) {
                                   inst[k] = i; len[k] = l; kind[k] = kd;
                                   if (geo) {
                                       for (int d = 0; d < 3; ++d) {
                                           geo[7 * k + d] = dv(p.r[d]);
                                           geo[7 * k + 3 + d] = dv(p.dir[d]);
                                       }
                                       geo[7 * k + 6] = dv(g->sigma[size_t(p.material)]);
                                   }
                               }
                               ++k;
                           });
    if (status) *status = h.status;
    return k;
}

// One history born at a given site, the way the power iteration births its
// later cycles from the bank (a bank of that one site): direction and tau
// from the particle's source counters, fission sites counted against knorm.
long long orc_trace_from_site(void* gp, long long pid, unsigned long long seed, double p_absorb, double knorm,
                              const double* site, long long cap, long long* inst, double* len, int* kind,
                              int* status) {
    Geometry* g = static_cast<Geometry*>(gp);
    RunOpts o;
    o.p_absorb = p_absorb;
    std::vector<uint64_t> tally(size_t(g->univ[g->root].ninst), 0);
    unsigned long long cnt[K_NCOUNTERS] = {0};
    const std::vector<double> bank(site, site + 3);
    long long k = 0;
    HistoryOut h = run_one(*g, uint32_t(pid), uint32_t(seed), o, tally.data(), cnt,
                           [&](long long i, double l, int kd, const Particle&) {
                               if (k < cap) { inst[k] = i; len[k] = l; kind[k] = kd; }
                               ++k;
                           }, nullptr, &bank, knorm);
    if (status) *status = h.status;
    return k;
}

// Hierarchical find_cell (Alg. 7) for global points: leaf instance or -1.
int orc_find_cell(void* gp, long long n, const double* xyz, long long* inst) {
    Geometry* g = static_cast<Geometry*>(gp);
    for (long long i = 0; i < n; ++i) {
        Particle p;
        for (int d = 0; d < 3; ++d) p.r[d] = xyz[3 * i + d];
        p.lv[0].u = g->root;
        inst[i] = find_cell_from(*g, p, 0) ? p.inst() : -1;
    }
    return 0;
}

// distance_to_surface (Table 1) from global points with directions, the
// point taken as on no surface: hierarchical find_cell, then the level scan
// of distance_to_boundary.  dist NaN and level/inst -1 for a point in no cell.
int orc_distance(void* gp, long long n, const double* xyz, const double* dir, double* dist, int* level,
                 long long* inst) {
    Geometry* g = static_cast<Geometry*>(gp);
    for (long long i = 0; i < n; ++i) {
        Particle p;
        for (int d = 0; d < 3; ++d) { p.r[d] = xyz[3 * i + d]; p.dir[d] = dir[3 * i + d]; }
        set_direction_inverse(p);
        p.lv[0].u = g->root;
        dist[i] = std::numeric_limits<double>::quiet_NaN();
        level[i] = -1;
        inst[i] = -1;
        if (!find_cell_from(*g, p, 0)) continue;
        const Hit h = distance_to_boundary(*g, p);
        dist[i] = dv(h.d);
        level[i] = h.level;
        inst[i] = p.inst();
    }
    return 0;
}

// Brute force over every leaf instance: first containing instance (-1 none),
// number of containing instances, and the distance from the point to the
// nearest constraint surface of any containing instance (or of all when none).
int orc_find_cell_brute(void* gp, long long n, const double* xyz, long long* inst, int* count, double* near) {
    Geometry* g = static_cast<Geometry*>(gp);
    std::vector<GLeaf> leaves;
    std::vector<GConstraint> chain;
    double T0[3] = {0, 0, 0};
    enumerate_leaves(*g, g->root, T0, chain, true, leaves);
    for (long long i = 0; i < n; ++i) {
        const double* x = xyz + 3 * i;
        inst[i] = -1;
        int cntv = 0;
        double nd = INF, nd_all = INF;
        for (size_t L = 0; L < leaves.size(); ++L) {
            bool in = true;
            double nl = INF;
            for (auto& k : leaves[L].cons) {
                double gr;
                double f = gc_f(k, x, &gr);
                nl = std::min(nl, std::fabs(f) / gr);
                int s = (k.type == S_CZ) ? ((f >= 0) ? 1 : -1) : ((f >= 0) ? 1 : -1);
                if (s != k.sense) in = false;
            }
            nd_all = std::min(nd_all, nl);
            if (in) { if (inst[i] < 0) inst[i] = (long long)L; ++cntv; nd = std::min(nd, nl); }
        }
        if (count) count[i] = cntv;
        if (near) near[i] = cntv ? nd : nd_all;
    }
    return int(leaves.size());
}

// Clearance of segments from the geometry's surfaces in the global frame,
// for telling whether a decision was taken close to a surface (test
// infrastructure: the tracking method itself never calls it).  Every leaf
// instance's constraint chain is moved into the global frame (as for the
// brute-force find_cell) and the distinct surfaces are kept.  For segment i
// (start xyz[3i..], unit direction dir[3i..], length len[i]):
//   out[8i+0], out[8i+1]  smallest distance from the start point to a
//                         surface (|f| / |grad f| for planes, |rho - r| for
//                         cylinders, rho the distance from the axis), and the
//                         smallest to any other surface
//   out[8i+2], out[8i+3]  the same at the end point xyz + len * dir
//   out[8i+4]             tangency: smallest |b - r| over the cylinders whose
//                         axis is closest to the segment's line (in the xy
//                         projection) at a point of the segment, b that
//                         closest distance; +inf when there is none
//   out[8i+5..7]          the unit normal n of the surface nearest to the
//                         end point, there (sign arbitrary; 0 when there is
//                         no surface)
int orc_clearance(void* gp, long long n, const double* xyz, const double* dir, const double* len, double* out) {
    Geometry* g = static_cast<Geometry*>(gp);
    std::vector<GLeaf> leaves;
    std::vector<GConstraint> chain;
    double T0[3] = {0, 0, 0};
    enumerate_leaves(*g, g->root, T0, chain, true, leaves);
    std::vector<GConstraint> surf;
    for (auto& L : leaves)
        for (auto& k : L.cons) surf.push_back(k);
    auto key_less = [](const GConstraint& a, const GConstraint& b) {
        if (a.type != b.type) return a.type < b.type;
        for (int i = 0; i < 4; ++i)
            if (a.c[i] != b.c[i]) return a.c[i] < b.c[i];
        return false;
    };
    auto key_eq = [](const GConstraint& a, const GConstraint& b) {
        if (a.type != b.type) return false;
        for (int i = 0; i < 4; ++i)
            if (a.c[i] != b.c[i]) return false;
        return true;
    };
    std::sort(surf.begin(), surf.end(), key_less);
    surf.erase(std::unique(surf.begin(), surf.end(), key_eq), surf.end());
    // The same physical surface can reach the list more than once with its
    // global coefficients rounded differently (a plane shared by cells of
    // different levels): the second distance skips every surface within
    // 1e-9 (relative to the coefficients' size) of the nearest one.
    auto same = [](const GConstraint& a, const GConstraint& b) {
        if (a.type != b.type) return false;
        for (int i = 0; i < 4; ++i)
            if (std::fabs(a.c[i] - b.c[i]) > 1e-9 * std::max(1.0, std::fabs(a.c[i]))) return false;
        return true;
    };
    auto two_smallest = [&](const double x[3], double& m1, double& m2, size_t* nearest = nullptr) {
        m1 = INF; m2 = INF;
        size_t best = 0;
        for (size_t i = 0; i < surf.size(); ++i) {
            double gr;
            const double d = std::fabs(gc_f(surf[i], x, &gr)) / gr;
            if (d < m1) { m1 = d; best = i; }
        }
        if (surf.empty()) return;
        if (nearest) *nearest = best;
        for (size_t i = 0; i < surf.size(); ++i) {
            if (same(surf[i], surf[best])) continue;
            double gr;
            m2 = std::min(m2, std::fabs(gc_f(surf[i], x, &gr)) / gr);
        }
    };
    for (long long i = 0; i < n; ++i) {
        const double* p = xyz + 3 * i;
        const double* w = dir + 3 * i;
        const double L = len[i];
        const double q[3] = {p[0] + L * w[0], p[1] + L * w[1], p[2] + L * w[2]};
        double* o6 = out + 8 * i;
        two_smallest(p, o6[0], o6[1]);
        size_t ns = surf.size();
        two_smallest(q, o6[2], o6[3], &ns);
        o6[5] = o6[6] = o6[7] = 0.0;
        if (ns < surf.size()) {
            const GConstraint& k = surf[ns];
            double nrm[3] = {0.0, 0.0, 0.0};
            if (k.type <= S_PZ) nrm[k.type] = 1.0;
            else if (k.type == S_P) {
                const double nn = std::sqrt(k.c[0] * k.c[0] + k.c[1] * k.c[1] + k.c[2] * k.c[2]);
                for (int d = 0; d < 3; ++d) nrm[d] = k.c[d] / nn;
            } else {
                const double qx = q[0] - k.c[0], qy = q[1] - k.c[1];
                const double rr = std::sqrt(qx * qx + qy * qy);
                if (rr > 0.0) { nrm[0] = qx / rr; nrm[1] = qy / rr; }
            }
            for (int d = 0; d < 3; ++d) o6[5 + d] = nrm[d];
        }
        double tang = INF;
        const double a = w[0] * w[0] + w[1] * w[1];
        if (a > 0.0) {
            for (auto& k : surf) {
                if (k.type != S_CZ) continue;
                const double qx = p[0] - k.c[0], qy = p[1] - k.c[1];
                const double ts = -(qx * w[0] + qy * w[1]) / a;
                if (!(ts >= 0.0 && ts <= L)) continue;
                const double cx = qx + ts * w[0], cy = qy + ts * w[1];
                tang = std::min(tang, std::fabs(std::sqrt(cx * cx + cy * cy) - k.c[2]));
            }
        }
        o6[4] = tang;
    }
    return int(surf.size());
}

int orc_transmission(void* gp, long long n, const double* rays, const double* sigma, double pitch,
                     double* T, double* lens, double* dT, unsigned long long* hash, int* status, int nthreads) {
    Geometry* g = static_cast<Geometry*>(gp);
    int nm = int(g->sigma.size());
    if (nthreads < 1) nthreads = 1;
    auto work = [&](int t) {
        long long lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
        for (long long i = lo; i < hi; ++i) {
            uint64_t hh;
            int st;
            transmit_one(*g, rays + 6 * i, sigma, pitch, T[i], lens + size_t(i) * nm,
                         dT ? dT + size_t(i) * (nm + NPARAM) : nullptr, hh, st);
            if (hash) hash[i] = hh;
            if (status) status[i] = st;
        }
    };
    if (nthreads == 1) work(0);
    else {
        std::vector<std::thread> th;
        for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
        for (auto& x : th) x.join();
    }
    return 0;
}

void orc_philox4x32_10(const unsigned* ctr, const unsigned* key, unsigned* out) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]}, k[2] = {key[0], key[1]}, o[4];
    philox4x32_10(c, k, o);
    for (int i = 0; i < 4; ++i) out[i] = o[i];
}

void orc_uniform2(unsigned pid, unsigned event, unsigned tag, unsigned k, unsigned seed_lo, unsigned gid, double* out) {
    uniform2(pid, event, tag, k, seed_lo, gid, out);
}

double orc_log(double x) { return dv(own_log(Real(x))); }

int orc_isotropic(unsigned pid, unsigned event, unsigned seed_lo, unsigned gid, double* dir) {
    Real d[3];
    bool ok = isotropic(pid, event, seed_lo, gid, d);
    for (int i = 0; i < 3; ++i) dir[i] = dv(d[i]);
    return ok ? 1 : 0;
}

// Operation counts (counting build only; zeros otherwise): add/sub, mul,
// div, sqrt, compare, accumulated by the calling thread since the last reset.
void orc_flop_counts(unsigned long long* out, int reset) {
#ifdef ORACLE_COUNT_FLOPS
    out[0] = g_fc.add; out[1] = g_fc.mul; out[2] = g_fc.div; out[3] = g_fc.sqrt; out[4] = g_fc.cmp;
    if (reset) g_fc = FlopCount{0, 0, 0, 0, 0};
#else
    (void)reset;
    for (int i = 0; i < 5; ++i) out[i] = 0;
#endif
}

int orc_counting_build(void) {
#ifdef ORACLE_COUNT_FLOPS
    return 1;
#else
    return 0;
#endif
}

}  // extern "C"
