// geometry_build.cpp - host side of the C-ABI: description parsing,
// pseudo-array conversion, cell boxes, SAH BVH, flattening to device memory.
//
// Paper: Sec. 1 (CSG cells as intersections of surface senses, universes
// nested in cells and arrays, Table 1), Sec. 3.2 (lower-level coincident
// boundary surfaces are removed), Sec. 4.3 (pseudo-array universes; cell
// boxes by truncating the universe box with the cell's bounding planes; SAH
// partitioning evaluating three equally spaced candidates per axis with a
// cost that balances box count and surface area).
//
// Compiled with -ffp-contract=off: the few floating-point values computed
// here that tracking uses (element centres, hex translations, plane offsets)
// are single IEEE operations, identical to any other IEEE evaluation.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <vector>

#include "trk.h"
#include "trk_internal.h"

namespace trk {

static thread_local std::string t_err;

int set_error(int st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

namespace {

const double INF = std::numeric_limits<double>::infinity();

// ---------------------------------------------------------------------------
// JSON: a flat node table filled by a recursive-descent scanner.
// ---------------------------------------------------------------------------
struct JNode {
    char t = 'n';                  // 'o' object, 'a' array, 'd' number, 's' string, 'b' bool, 'n' null
    double d = 0;
    std::string s;
    std::vector<std::string> keys; // object keys (parallel to kids)
    std::vector<int> kids;
};

class Json {
  public:
    std::vector<JNode> nodes;
    std::string err;
    bool parse(const char* b, size_t n) {
        p_ = b; e_ = b + n;
        int root = value();
        if (root < 0) return false;
        skip();
        if (p_ != e_) { err = "trailing characters after JSON value"; return false; }
        return true;
    }
    const JNode& at(int i) const { return nodes[size_t(i)]; }
    int member(int obj, const char* k) const {
        const JNode& o = at(obj);
        if (o.t != 'o') return -1;
        for (size_t i = 0; i < o.keys.size(); ++i) if (o.keys[i] == k) return o.kids[i];
        return -1;
    }

  private:
    const char* p_ = nullptr;
    const char* e_ = nullptr;
    void skip() { while (p_ < e_ && (*p_ == ' ' || *p_ == '\t' || *p_ == '\n' || *p_ == '\r')) ++p_; }
    int bad(const char* m) { if (err.empty()) err = m; return -1; }
    int add(JNode&& n) { nodes.push_back(std::move(n)); return int(nodes.size()) - 1; }
    bool str(std::string& out) {
        if (p_ >= e_ || *p_ != '"') return false;
        ++p_;
        while (p_ < e_ && *p_ != '"') {
            if (*p_ == '\\' && p_ + 1 < e_) ++p_;
            out.push_back(*p_++);
        }
        if (p_ >= e_) return false;
        ++p_;
        return true;
    }
    int depth_ = 0;
    static const int MAX_DEPTH = 64;   // descriptions nest about five deep; this bounds the recursion
    int value() {
        if (depth_ >= MAX_DEPTH) return bad("JSON nested too deeply");
        ++depth_;
        const int v = value_at();
        --depth_;
        return v;
    }
    int value_at() {
        skip();
        if (p_ >= e_) return bad("unexpected end of description");
        if (*p_ == '{') {
            ++p_;
            int self = add(JNode{});
            nodes[size_t(self)].t = 'o';
            skip();
            if (p_ < e_ && *p_ == '}') { ++p_; return self; }
            while (true) {
                skip();
                std::string k;
                if (!str(k)) return bad("expected object key");
                skip();
                if (p_ >= e_ || *p_ != ':') return bad("expected ':'");
                ++p_;
                int v = value();
                if (v < 0) return -1;
                nodes[size_t(self)].keys.push_back(k);
                nodes[size_t(self)].kids.push_back(v);
                skip();
                if (p_ < e_ && *p_ == ',') { ++p_; continue; }
                if (p_ < e_ && *p_ == '}') { ++p_; return self; }
                return bad("expected ',' or '}'");
            }
        }
        if (*p_ == '[') {
            ++p_;
            int self = add(JNode{});
            nodes[size_t(self)].t = 'a';
            skip();
            if (p_ < e_ && *p_ == ']') { ++p_; return self; }
            while (true) {
                int v = value();
                if (v < 0) return -1;
                nodes[size_t(self)].kids.push_back(v);
                skip();
                if (p_ < e_ && *p_ == ',') { ++p_; continue; }
                if (p_ < e_ && *p_ == ']') { ++p_; return self; }
                return bad("expected ',' or ']'");
            }
        }
        JNode n;
        if (*p_ == '"') {
            n.t = 's';
            if (!str(n.s)) return bad("unterminated string");
            return add(std::move(n));
        }
        static const char* lits[3] = {"true", "false", "null"};
        for (int i = 0; i < 3; ++i) {
            size_t L = std::strlen(lits[i]);
            if (size_t(e_ - p_) >= L && std::strncmp(p_, lits[i], L) == 0) {
                p_ += L;
                n.t = i < 2 ? 'b' : 'n';
                n.d = (i == 0) ? 1.0 : 0.0;
                return add(std::move(n));
            }
        }
        char tmp[64];
        size_t k = 0;
        while (p_ < e_ && k < sizeof tmp - 1 && (std::isdigit((unsigned char)*p_) || *p_ == '-' || *p_ == '+' ||
                                                *p_ == '.' || *p_ == 'e' || *p_ == 'E'))
            tmp[k++] = *p_++;
        tmp[k] = 0;
        if (k == 0) return bad("unexpected character in description");
        char* end = nullptr;
        n.t = 'd';
        n.d = std::strtod(tmp, &end);
        if (end != tmp + k) return bad("malformed number");
        return add(std::move(n));
    }
};

// ---------------------------------------------------------------------------
// Host model
// ---------------------------------------------------------------------------
enum { UT_CSG = 0, UT_RECT = 1, UT_HEX = 2 };

struct HSurf {
    int type = 0;
    double c[4] = {0, 0, 0, 0};
    int bc = BC_NONE, rparam = -1, pscale = 0;
};
struct HCell {
    std::vector<int> surf, sense;
    int fill = -1;        // >= 0 daughter universe; < 0 material ~fill
    double tr[3] = {0, 0, 0};
    long long off = 0;
    double box[6] = {-INF, -INF, -INF, INF, INF, INF};
};
struct HUniv {
    int type = UT_CSG;
    std::vector<HCell> cells;   // CSG cells; pseudo-array cells for arrays
    std::vector<double> grid[3];
    int rings = 0;
    double a1[2] = {0, 0}, a2[2] = {0, 0}, nrm[3][2] = {{0, 0}, {0, 0}, {0, 0}}, hp = 0, z[2] = {0, 0};
    std::vector<int> hq, hr, fill;
    std::vector<long long> eoff;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    int pscale = 0;
    long long ninst = -1;
    double box[6] = {INF, INF, INF, -INF, -INF, -INF};   // universe box (own frame), grown from parents
    bool box_set = false;
    int first_cell = 0, bvh = -1, bih = -1, lat = -1;
};
struct HGeom {
    std::vector<double> mesh[3];   // superimposed mesh planes (empty: none)
    int accel = 0;                 // CSG cell search: 0 BVH, 1 BIH
    int gid = 0;
    std::vector<double> sigma;
    std::vector<double> nu;
    std::vector<HSurf> surf;
    std::vector<HUniv> univ;
    int root = 0;
    double src[6] = {0, 0, 0, 0, 0, 0};
    int depth = 0;
    bool rect_ok = true;
};

int bc_code(const Json& J, int node) {
    if (node < 0 || J.at(node).t != 's') return BC_NONE;
    const std::string& s = J.at(node).s;
    if (s == "vacuum") return BC_VACUUM;
    if (s == "reflect") return BC_REFLECT;
    return BC_NONE;
}

bool read_nums(const Json& J, int node, std::vector<double>& out) {
    out.clear();
    if (node < 0 || J.at(node).t != 'a') return false;
    for (int k : J.at(node).kids) {
        if (J.at(k).t != 'd') return false;
        out.push_back(J.at(k).d);
    }
    return true;
}

bool finite_all(const std::vector<double>& v) {
    for (double x : v) if (!std::isfinite(x)) return false;
    return true;
}

bool num(const Json& J, int obj, const char* key, double& out) {
    int m = J.member(obj, key);
    if (m < 0 || J.at(m).t != 'd') return false;
    out = J.at(m).d;
    return true;
}

// Optional integer member: absent leaves `out` as it is; present, it must be
// a number holding an integer in [lo, hi].
bool opt_int(const Json& J, int obj, const char* key, int lo, int hi, int& out) {
    int m = J.member(obj, key);
    if (m < 0) return true;
    if (J.at(m).t != 'd') return false;
    const double v = J.at(m).d;
    if (!(v >= double(lo) && v <= double(hi)) || v != std::floor(v)) return false;
    out = int(v);
    return true;
}

#define DESC_FAIL(...) return set_error(TRK_E_DESC, __VA_ARGS__)

int parse(const char* json, size_t len, HGeom& G) {
    Json J;
    if (!J.parse(json, len)) DESC_FAIL("description JSON: %s", J.err.c_str());
    const int root = 0;
    if (J.at(root).t != 'o') DESC_FAIL("description is not a JSON object");
    double x;
    if (!opt_int(J, root, "geometry_id", 0, 0x7fffffff, G.gid)) DESC_FAIL("'geometry_id' must be an integer in [0, 2^31)");
    if (!read_nums(J, J.member(root, "sigma"), G.sigma) || G.sigma.empty()) DESC_FAIL("'sigma' missing or empty");
    for (double s : G.sigma) if (!(s >= 0.0) || !std::isfinite(s)) DESC_FAIL("sigma must be finite and >= 0");
    G.nu.assign(G.sigma.size(), 0.0);
    if (J.member(root, "nu") >= 0) {
        if (!read_nums(J, J.member(root, "nu"), G.nu) || G.nu.size() != G.sigma.size()) DESC_FAIL("'nu' needs one value per material");
        for (double v : G.nu) if (!(v >= 0.0 && v <= 7.0)) DESC_FAIL("nu must be in [0, 7]");
    }
    int sl = J.member(root, "surfaces");
    if (sl < 0 || J.at(sl).t != 'a') DESC_FAIL("'surfaces' missing");
    for (size_t i = 0; i < J.at(sl).kids.size(); ++i) {
        int so = J.at(sl).kids[i];
        HSurf s;
        int tn = J.member(so, "type");
        std::vector<double> cf;
        if (tn < 0 || J.at(tn).t != 's' || !read_nums(J, J.member(so, "coef"), cf)) DESC_FAIL("surface %zu malformed", i);
        const std::string& t = J.at(tn).s;
        size_t need = 0;
        if (t == "px") { s.type = S_PX; need = 1; }
        else if (t == "py") { s.type = S_PY; need = 1; }
        else if (t == "pz") { s.type = S_PZ; need = 1; }
        else if (t == "p") { s.type = S_P; need = 4; }
        else if (t == "cz") { s.type = S_CZ; need = 3; }
        else DESC_FAIL("surface %zu: unknown type '%s'", i, t.c_str());
        if (cf.size() != need) DESC_FAIL("surface %zu: expected %zu coefficients", i, need);
        for (size_t k = 0; k < need; ++k) {
            if (!std::isfinite(cf[k])) DESC_FAIL("surface %zu: non-finite coefficient", i);
            s.c[k] = cf[k];
        }
        if (s.type == S_CZ && !(s.c[2] > 0)) DESC_FAIL("surface %zu: cylinder radius must be > 0", i);
        s.bc = bc_code(J, J.member(so, "bc"));
        if (s.bc == BC_REFLECT && s.type == S_CZ) DESC_FAIL("surface %zu: reflecting cylinders are not supported", i);
        if (!opt_int(J, so, "rparam", -1, TRK_NGEOM_PARAMS - 2, s.rparam)) DESC_FAIL("surface %zu: 'rparam' must be -1, 0, 1 or 2", i);
        if (!opt_int(J, so, "pscale", 0, 1, s.pscale)) DESC_FAIL("surface %zu: 'pscale' must be 0 or 1", i);
        G.surf.push_back(s);
    }
    int ul = J.member(root, "universes");
    if (ul < 0 || J.at(ul).t != 'a' || J.at(ul).kids.empty()) DESC_FAIL("'universes' missing or empty");
    const int nu = int(J.at(ul).kids.size());
    for (int ui = 0; ui < nu; ++ui) {
        int uo = J.at(ul).kids[size_t(ui)];
        HUniv U;
        int tn = J.member(uo, "type");
        if (tn < 0 || J.at(tn).t != 's') DESC_FAIL("universe %d: missing type", ui);
        const std::string& t = J.at(tn).s;
        if (t == "csg") {
            U.type = UT_CSG;
            int cl = J.member(uo, "cells");
            if (cl < 0 || J.at(cl).t != 'a' || J.at(cl).kids.empty()) DESC_FAIL("universe %d: csg needs cells", ui);
            for (size_t ci = 0; ci < J.at(cl).kids.size(); ++ci) {
                int co = J.at(cl).kids[ci];
                HCell c;
                int ss = J.member(co, "surfaces");
                if (ss < 0 || J.at(ss).t != 'a') DESC_FAIL("universe %d cell %zu: missing surfaces", ui, ci);
                for (int pr : J.at(ss).kids) {
                    std::vector<double> v;
                    if (!read_nums(J, pr, v) || v.size() != 2) DESC_FAIL("universe %d cell %zu: bad surface pair", ui, ci);
                    if (!(v[0] >= 0.0 && v[0] < double(G.surf.size())) || v[0] != std::floor(v[0]))
                        DESC_FAIL("universe %d cell %zu: bad surface id", ui, ci);
                    if (v[1] != 1.0 && v[1] != -1.0) DESC_FAIL("universe %d cell %zu: sense must be +1 or -1", ui, ci);
                    const int sid = int(v[0]), sn = int(v[1]);
                    c.surf.push_back(sid);
                    c.sense.push_back(sn);
                }
                double m;
                if (num(J, co, "material", m)) {
                    if (m < 0 || m >= double(G.sigma.size()) || double(int(m)) != m) DESC_FAIL("universe %d cell %zu: bad material", ui, ci);
                    c.fill = ~int(m);
                } else if (num(J, co, "fill", m)) {
                    if (m < 0 || m >= nu || double(int(m)) != m) DESC_FAIL("universe %d cell %zu: bad fill", ui, ci);
                    c.fill = int(m);
                    std::vector<double> tr;
                    int tn2 = J.member(co, "translation");
                    if (tn2 >= 0) {
                        if (!read_nums(J, tn2, tr) || tr.size() != 3 || !finite_all(tr)) DESC_FAIL("universe %d cell %zu: bad translation", ui, ci);
                        for (int d = 0; d < 3; ++d) c.tr[d] = tr[size_t(d)];
                    }
                } else DESC_FAIL("universe %d cell %zu: needs 'material' or 'fill'", ui, ci);
                U.cells.push_back(c);
            }
        } else if (t == "rect") {
            U.type = UT_RECT;
            int gl = J.member(uo, "grid");
            if (gl < 0 || J.at(gl).t != 'a' || J.at(gl).kids.size() != 3) DESC_FAIL("universe %d: rect needs 3 grids", ui);
            size_t ne = 1;
            for (int d = 0; d < 3; ++d) {
                if (!read_nums(J, J.at(gl).kids[size_t(d)], U.grid[d]) || U.grid[d].size() < 2 || !finite_all(U.grid[d]))
                    DESC_FAIL("universe %d: bad grid %d", ui, d);
                for (size_t i = 1; i < U.grid[d].size(); ++i)
                    if (!(U.grid[d][i] > U.grid[d][i - 1])) DESC_FAIL("universe %d: grid %d not increasing", ui, d);
                ne *= U.grid[d].size() - 1;
            }
            std::vector<double> fl;
            if (!read_nums(J, J.member(uo, "fill"), fl) || fl.size() != ne) DESC_FAIL("universe %d: fill needs %zu entries", ui, ne);
            for (double f : fl) {
                if (f < 0 || f >= nu || double(int(f)) != f) DESC_FAIL("universe %d: bad fill entry", ui);
                U.fill.push_back(int(f));
            }
            int bl = J.member(uo, "bc");
            if (bl >= 0) {
                if (J.at(bl).t != 'a' || J.at(bl).kids.size() != 6) DESC_FAIL("universe %d: rect bc needs 6 entries", ui);
                for (int k = 0; k < 6; ++k) U.bc[k] = bc_code(J, J.at(bl).kids[size_t(k)]);
            }
            if (!opt_int(J, uo, "pscale", 0, 1, U.pscale)) DESC_FAIL("universe %d: 'pscale' must be 0 or 1", ui);
        } else if (t == "hex") {
            U.type = UT_HEX;
            std::vector<double> a1, a2, zz;
            double rings, hp;
            if (!num(J, uo, "rings", rings) || !(rings >= 0 && rings <= 64) || rings != std::floor(rings) || !read_nums(J, J.member(uo, "a1"), a1) ||
                !read_nums(J, J.member(uo, "a2"), a2) || !read_nums(J, J.member(uo, "z"), zz) || a1.size() != 2 ||
                a2.size() != 2 || zz.size() != 2 || !num(J, uo, "half_pitch", hp) || !(hp > 0) || !std::isfinite(hp) ||
                !finite_all(a1) || !finite_all(a2) || !finite_all(zz) || !(zz[1] > zz[0]))
                DESC_FAIL("universe %d: malformed hex array", ui);
            U.rings = int(rings);
            U.a1[0] = a1[0]; U.a1[1] = a1[1]; U.a2[0] = a2[0]; U.a2[1] = a2[1];
            U.z[0] = zz[0]; U.z[1] = zz[1]; U.hp = hp;
            if (!(std::fabs(a1[0] * a2[1] - a2[0] * a1[1]) > 0)) DESC_FAIL("universe %d: hex lattice vectors are parallel", ui);
            int nl = J.member(uo, "normals");
            if (nl < 0 || J.at(nl).t != 'a' || J.at(nl).kids.size() != 3) DESC_FAIL("universe %d: hex needs 3 normals", ui);
            for (int k = 0; k < 3; ++k) {
                std::vector<double> nk;
                if (!read_nums(J, J.at(nl).kids[size_t(k)], nk) || nk.size() != 2 || !finite_all(nk) || !(nk[0] != 0.0 || nk[1] != 0.0))
                    DESC_FAIL("universe %d: bad hex normal", ui);
                U.nrm[k][0] = nk[0]; U.nrm[k][1] = nk[1];
            }
            const int R = U.rings;
            for (int r = -R; r <= R; ++r)
                for (int q = std::max(-R, -R - r); q <= std::min(R, R - r); ++q) { U.hq.push_back(q); U.hr.push_back(r); }
            std::vector<double> fl;
            if (!read_nums(J, J.member(uo, "fill"), fl) || fl.size() != U.hq.size()) DESC_FAIL("universe %d: hex fill needs %zu entries", ui, U.hq.size());
            for (double f : fl) {
                if (f < 0 || f >= nu || double(int(f)) != f) DESC_FAIL("universe %d: bad fill entry", ui);
                U.fill.push_back(int(f));
            }
            int bl = J.member(uo, "bc");
            if (bl >= 0) {
                if (J.at(bl).t != 'a' || J.at(bl).kids.size() != 3) DESC_FAIL("universe %d: hex bc needs 3 entries", ui);
                U.bc[0] = bc_code(J, J.at(bl).kids[0]);
                U.bc[4] = bc_code(J, J.at(bl).kids[1]);
                U.bc[5] = bc_code(J, J.at(bl).kids[2]);
            }
        } else DESC_FAIL("universe %d: unknown type '%s'", ui, t.c_str());
        G.univ.push_back(std::move(U));
    }
    if (!num(J, root, "root", x) || x < 0 || x >= nu || double(int(x)) != x) DESC_FAIL("'root' missing or out of range");
    G.root = int(x);
    std::vector<double> sb;
    if (!read_nums(J, J.member(root, "source_box"), sb) || sb.size() != 6 || !finite_all(sb)) DESC_FAIL("'source_box' needs 6 finite numbers");
    {
        const int ao = J.member(root, "accel");
        if (ao >= 0) {
            if (J.at(ao).t != 's' || (J.at(ao).s != "bvh" && J.at(ao).s != "bih")) DESC_FAIL("'accel' must be \"bvh\" or \"bih\"");
            G.accel = J.at(ao).s == "bih" ? 1 : 0;
        }
    }
    {
        const int mo = J.member(root, "mesh");
        if (mo >= 0) {
            const int mg = J.member(mo, "grid");
            if (mg < 0 || J.at(mg).t != 'a' || J.at(mg).kids.size() != 3) DESC_FAIL("'mesh' needs 3 grids");
            long long bins = 1;
            for (int d = 0; d < 3; ++d) {
                if (!read_nums(J, J.at(mg).kids[size_t(d)], G.mesh[d]) || G.mesh[d].size() < 2) DESC_FAIL("mesh grid %d malformed", d);
                for (size_t i = 0; i < G.mesh[d].size(); ++i) {
                    if (!std::isfinite(G.mesh[d][i])) DESC_FAIL("mesh grid %d: non-finite plane", d);
                    if (i > 0 && !(G.mesh[d][i] > G.mesh[d][i - 1])) DESC_FAIL("mesh grid %d not increasing", d);
                }
                bins *= (long long)(G.mesh[d].size() - 1);
            }
            if (bins > (1LL << 31)) DESC_FAIL("mesh has more than 2^31 bins");
        }
    }
    for (int k = 0; k < 3; ++k) if (!(sb[size_t(k + 3)] > sb[size_t(k)])) DESC_FAIL("'source_box' is empty");
    for (int k = 0; k < 6; ++k) G.src[k] = sb[size_t(k)];
    return TRK_OK;
}

// Leaf-instance counts and offsets (cells in order; array elements i fastest,
// hex rows r = -R..R with q ascending), memoised per universe, with the
// height of each universe's subtree; a universe reached again while still
// being counted means a cycle.
int count_instances(HGeom& G, int u, std::vector<int>& height, std::vector<char>& busy) {
    HUniv& U = G.univ[size_t(u)];
    if (U.ninst >= 0) return TRK_OK;
    if (busy[size_t(u)]) return set_error(TRK_E_DESC, "universe %d contains itself", u);
    busy[size_t(u)] = 1;
    long long total = 0;
    int h = 0;
    auto child = [&](int d) -> int {
        int st = count_instances(G, d, height, busy);
        if (st != TRK_OK) return st;
        h = std::max(h, height[size_t(d)] + 1);
        total += G.univ[size_t(d)].ninst;
        return TRK_OK;
    };
    if (U.type == UT_CSG) {
        for (auto& c : U.cells) {
            c.off = total;
            if (c.fill < 0) total += 1;
            else if (int st = child(c.fill)) return st;
        }
    } else {
        U.eoff.assign(U.fill.size(), 0);
        for (size_t e = 0; e < U.fill.size(); ++e) {
            U.eoff[e] = total;
            if (int st = child(U.fill[e])) return st;
        }
    }
    busy[size_t(u)] = 0;
    U.ninst = total;
    height[size_t(u)] = h;
    if (total > (1LL << 31) - 1) return set_error(TRK_E_DESC, "more than 2^31-1 leaf cell instances");
    return TRK_OK;
}

// Sec. 4.3 pseudo-array: one CSG cell per element, faces in the order
// (dim 0 lower, dim 0 upper, dim 1 lower, ...), outer faces of a non-root
// array left out (Sec. 3.2: the parent level owns that boundary).
void make_pseudo_array(HGeom& G, int u) {
    HUniv& U = G.univ[size_t(u)];
    const bool is_root = (u == G.root);
    U.cells.clear();
    if (U.type == UT_RECT) {
        int n[3];
        std::vector<int> sid[3];
        for (int d = 0; d < 3; ++d) {
            n[d] = int(U.grid[d].size()) - 1;
            for (int i = 0; i <= n[d]; ++i) {
                HSurf s;
                s.type = d;
                s.c[0] = U.grid[d][size_t(i)];
                s.pscale = d < 2 ? U.pscale : 0;
                if (i == 0) s.bc = U.bc[2 * d];
                if (i == n[d]) s.bc = U.bc[2 * d + 1];
                sid[d].push_back(int(G.surf.size()));
                G.surf.push_back(s);
            }
        }
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    HCell c;
                    const int ijk[3] = {i, j, k};
                    for (int d = 0; d < 3; ++d) {
                        if (is_root || ijk[d] > 0) { c.surf.push_back(sid[d][size_t(ijk[d])]); c.sense.push_back(+1); }
                        if (is_root || ijk[d] < n[d] - 1) { c.surf.push_back(sid[d][size_t(ijk[d] + 1)]); c.sense.push_back(-1); }
                    }
                    size_t e = size_t(i + n[0] * (j + n[1] * k));
                    c.fill = U.fill[e];
                    c.off = U.eoff[e];
                    c.tr[0] = (U.grid[0][size_t(i)] + U.grid[0][size_t(i) + 1]) * 0.5;
                    c.tr[1] = (U.grid[1][size_t(j)] + U.grid[1][size_t(j) + 1]) * 0.5;
                    c.tr[2] = (U.grid[2][size_t(k)] + U.grid[2][size_t(k) + 1]) * 0.5;
                    U.cells.push_back(c);
                }
        return;
    }
    // hex: face planes of family f are nrm_f . x = j * half_pitch; element
    // (q, r) is bounded by j = m_f - 1 (its + side) and m_f + 1 (its - side)
    // with m = (2q + r, q + 2r, r - q); one surface per (f, j).
    std::map<std::pair<int, int>, int> planes;
    auto plane = [&](int f, int j) {
        auto it = planes.find({f, j});
        if (it != planes.end()) return it->second;
        HSurf s;
        s.type = S_P;
        s.c[0] = U.nrm[f][0];
        s.c[1] = U.nrm[f][1];
        s.c[2] = 0.0;
        s.c[3] = double(j) * U.hp;
        s.bc = U.bc[0];
        int id = int(G.surf.size());
        G.surf.push_back(s);
        planes[{f, j}] = id;
        return id;
    };
    int zs[2] = {-1, -1};
    if (is_root)
        for (int t = 0; t < 2; ++t) {
            HSurf s;
            s.type = S_PZ;
            s.c[0] = U.z[t];
            s.bc = U.bc[4 + t];
            zs[t] = int(G.surf.size());
            G.surf.push_back(s);
        }
    std::map<std::pair<int, int>, int> where;
    for (size_t e = 0; e < U.hq.size(); ++e) where[{U.hq[e], U.hr[e]}] = int(e);
    for (size_t e = 0; e < U.hq.size(); ++e) {
        const int q = U.hq[e], r = U.hr[e];
        const int m[3] = {2 * q + r, q + 2 * r, r - q};
        const int lo_nb[3][2] = {{q - 1, r}, {q, r - 1}, {q + 1, r - 1}};
        const int hi_nb[3][2] = {{q + 1, r}, {q, r + 1}, {q - 1, r + 1}};
        HCell c;
        for (int f = 0; f < 3; ++f) {
            if (is_root || where.count({lo_nb[f][0], lo_nb[f][1]})) { c.surf.push_back(plane(f, m[f] - 1)); c.sense.push_back(+1); }
            if (is_root || where.count({hi_nb[f][0], hi_nb[f][1]})) { c.surf.push_back(plane(f, m[f] + 1)); c.sense.push_back(-1); }
        }
        if (is_root) {
            c.surf.push_back(zs[0]); c.sense.push_back(+1);
            c.surf.push_back(zs[1]); c.sense.push_back(-1);
        }
        c.fill = U.fill[e];
        c.off = U.eoff[e];
        const double qd = double(q), rd = double(r);
        c.tr[0] = qd * U.a1[0] + rd * U.a2[0];
        c.tr[1] = qd * U.a1[1] + rd * U.a2[1];
        c.tr[2] = (U.z[0] + U.z[1]) * 0.5;
        U.cells.push_back(c);
    }
}

// ---------------------------------------------------------------------------
// Cell boxes (Sec. 4.3): start from the universe box and truncate by each of
// the cell's surfaces; slanted planes clip the xy polygon of the box.
// ---------------------------------------------------------------------------
void clip_polygon(std::vector<std::pair<double, double>>& poly, double nx, double ny, double d, int sense) {
    // keep sense * (n.x - d) >= 0
    std::vector<std::pair<double, double>> out;
    const size_t n = poly.size();
    for (size_t i = 0; i < n; ++i) {
        auto a = poly[i], b = poly[(i + 1) % n];
        double fa = sense * (nx * a.first + ny * a.second - d);
        double fb = sense * (nx * b.first + ny * b.second - d);
        if (fa >= 0) out.push_back(a);
        if ((fa >= 0) != (fb >= 0)) {
            double t = fa / (fa - fb);
            out.push_back({a.first + t * (b.first - a.first), a.second + t * (b.second - a.second)});
        }
    }
    poly.swap(out);
}

void cell_box(const HGeom& G, const HUniv& U, HCell& c) {
    double b[6];
    for (int k = 0; k < 6; ++k) b[k] = U.box[k];
    std::vector<int> slanted;
    for (size_t i = 0; i < c.surf.size(); ++i) {
        const HSurf& s = G.surf[size_t(c.surf[i])];
        const int sn = c.sense[i];
        if (s.type <= S_PZ) {
            if (sn > 0) b[s.type] = std::max(b[s.type], s.c[0]);
            else b[3 + s.type] = std::min(b[3 + s.type], s.c[0]);
        } else if (s.type == S_CZ) {
            if (sn < 0) {
                b[0] = std::max(b[0], s.c[0] - s.c[2]);
                b[3] = std::min(b[3], s.c[0] + s.c[2]);
                b[1] = std::max(b[1], s.c[1] - s.c[2]);
                b[4] = std::min(b[4], s.c[1] + s.c[2]);
            }
        } else if (s.c[2] == 0.0) {
            slanted.push_back(int(i));
        }
    }
    if (!slanted.empty()) {
        // Clip a square sized from the cell's own numbers (not a huge one:
        // polygon vertices computed near 1e12 lose ~1e-4 to cancellation).
        // A cell that still reaches the square's edge is unbounded there.
        double S = 1.0;
        for (int i : slanted) S = std::max(S, std::fabs(G.surf[size_t(c.surf[size_t(i)])].c[3]));
        for (int k : {0, 1, 3, 4}) if (std::isfinite(b[k])) S = std::max(S, std::fabs(b[k]));
        S = 4.0 * S + 1.0;
        double x0 = std::max(b[0], -S), x1 = std::min(b[3], S);
        double y0 = std::max(b[1], -S), y1 = std::min(b[4], S);
        std::vector<std::pair<double, double>> poly = {{x0, y0}, {x1, y0}, {x1, y1}, {x0, y1}};
        for (int i : slanted) {
            const HSurf& s = G.surf[size_t(c.surf[size_t(i)])];
            clip_polygon(poly, s.c[0], s.c[1], s.c[3], c.sense[size_t(i)]);
            if (poly.empty()) break;
        }
        if (poly.empty()) {
            b[3] = b[0]; b[4] = b[1];   // empty in xy: keep a degenerate box
        } else {
            double px0 = INF, px1 = -INF, py0 = INF, py1 = -INF;
            for (auto& p : poly) {
                px0 = std::min(px0, p.first); px1 = std::max(px1, p.first);
                py0 = std::min(py0, p.second); py1 = std::max(py1, p.second);
            }
            const double edge = S * (1.0 - 1e-9);
            b[0] = (px0 <= -edge && !std::isfinite(b[0])) ? -INF : px0;
            b[3] = (px1 >= edge && !std::isfinite(b[3])) ? INF : px1;
            b[1] = (py0 <= -edge && !std::isfinite(b[1])) ? -INF : py0;
            b[4] = (py1 >= edge && !std::isfinite(b[4])) ? INF : py1;
        }
    }
    for (int k = 0; k < 6; ++k) c.box[k] = b[k];
}

// Boxes padded outward by 2^-40 max(1,|v|) plus a polygon-clipping margin.
void pad_box(double* b) {
    for (int k = 0; k < 3; ++k) {
        if (std::isfinite(b[k])) b[k] -= std::ldexp(std::max(1.0, std::fabs(b[k])), -40) + 1e-9;
        if (std::isfinite(b[3 + k])) b[3 + k] += std::ldexp(std::max(1.0, std::fabs(b[3 + k])), -40) + 1e-9;
    }
}

// Universe boxes top-down (each universe: union over its uses of the
// parent cell's box, moved into the universe's frame), then cell boxes.
void compute_boxes(HGeom& G) {
    const int nu = int(G.univ.size());
    // topological order from the root (the universe graph is a DAG)
    std::vector<int> indeg(size_t(nu), 0), order;
    std::vector<char> reach(size_t(nu), 0);
    std::vector<int> stack = {G.root};
    reach[size_t(G.root)] = 1;
    while (!stack.empty()) {
        int u = stack.back();
        stack.pop_back();
        for (auto& c : G.univ[size_t(u)].cells)
            if (c.fill >= 0 && !reach[size_t(c.fill)]) { reach[size_t(c.fill)] = 1; stack.push_back(c.fill); }
    }
    for (int u = 0; u < nu; ++u)
        if (reach[size_t(u)])
            for (auto& c : G.univ[size_t(u)].cells) if (c.fill >= 0) indeg[size_t(c.fill)]++;
    std::vector<int> q = {G.root};
    while (!q.empty()) {
        int u = q.back();
        q.pop_back();
        order.push_back(u);
        for (auto& c : G.univ[size_t(u)].cells)
            if (c.fill >= 0 && --indeg[size_t(c.fill)] == 0) q.push_back(c.fill);
    }
    HUniv& R = G.univ[size_t(G.root)];
    for (int k = 0; k < 3; ++k) { R.box[k] = -INF; R.box[3 + k] = INF; }
    R.box_set = true;
    for (int u : order) {
        HUniv& U = G.univ[size_t(u)];
        if (!U.box_set) for (int k = 0; k < 3; ++k) { U.box[k] = -INF; U.box[3 + k] = INF; }
        for (auto& c : U.cells) {
            cell_box(G, U, c);
            if (c.fill >= 0) {
                HUniv& D = G.univ[size_t(c.fill)];
                for (int k = 0; k < 3; ++k) {
                    double lo = c.box[k] - c.tr[k], hi = c.box[3 + k] - c.tr[k];
                    if (!D.box_set) { D.box[k] = lo; D.box[3 + k] = hi; }
                    else { D.box[k] = std::min(D.box[k], lo); D.box[3 + k] = std::max(D.box[3 + k], hi); }
                }
                D.box_set = true;
            }
            pad_box(c.box);
        }
    }
}

// ---------------------------------------------------------------------------
// SAH BVH over cell boxes (Sec. 4.3: three equally spaced candidate planes
// per axis on the box centres; cost = n_L * area(L) + n_R * area(R)).
// ---------------------------------------------------------------------------
struct Box { double lo[3], hi[3]; };

float f_down(double v) {
    if (v == -INF) return -std::numeric_limits<float>::infinity();
    if (v >= 3.0e38) return std::numeric_limits<float>::max();
    float f = float(v);
    if (double(f) > v) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}
float f_up(double v) {
    if (v == INF) return std::numeric_limits<float>::infinity();
    if (v <= -3.0e38) return -std::numeric_limits<float>::max();
    float f = float(v);
    if (double(f) < v) f = std::nextafter(f, std::numeric_limits<float>::infinity());
    return f;
}

class BvhBuilder {
  public:
    std::vector<BvhNode> nodes;
    std::vector<int> leaf_cells;
    int max_depth = 0;
    Box proxy;   // finite stand-in for infinite extents in the cost

    // Builds the tree over `cells` and returns its root reference (a node
    // index, or a leaf reference for a universe of at most BVH_LEAF_MAX cells).
    int build(std::vector<int>& cells, const std::vector<Box>& boxes) {
        ids_ = cells;
        boxes_ = &boxes;
        return emit(0, int(ids_.size()), 0);
    }

  private:
    std::vector<int> ids_;
    const std::vector<Box>* boxes_ = nullptr;

    double clampv(double v, int k) const { return std::min(std::max(v, proxy.lo[k]), proxy.hi[k]); }
    double centre(int id, int k) const {
        const Box& b = (*boxes_)[size_t(id)];
        return 0.5 * (clampv(b.lo[k], k) + clampv(b.hi[k], k));
    }
    Box bound(int lo, int hi) const {
        Box r;
        for (int k = 0; k < 3; ++k) { r.lo[k] = INF; r.hi[k] = -INF; }
        for (int i = lo; i < hi; ++i) {
            const Box& b = (*boxes_)[size_t(ids_[size_t(i)])];
            for (int k = 0; k < 3; ++k) { r.lo[k] = std::min(r.lo[k], b.lo[k]); r.hi[k] = std::max(r.hi[k], b.hi[k]); }
        }
        return r;
    }
    double area(const Box& b) const {
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = std::max(0.0, clampv(b.hi[k], k) - clampv(b.lo[k], k));
        return 2.0 * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0]);
    }
    // SAH split of [lo, hi): three equally spaced candidate planes per axis on
    // the box centres, cost n_L area(L) + n_R area(R); median if none splits.
    int split(int lo, int hi) {
        const int n = hi - lo;
        double cmin[3], cmax[3];
        for (int k = 0; k < 3; ++k) { cmin[k] = INF; cmax[k] = -INF; }
        for (int i = lo; i < hi; ++i)
            for (int k = 0; k < 3; ++k) {
                double c = centre(ids_[size_t(i)], k);
                cmin[k] = std::min(cmin[k], c); cmax[k] = std::max(cmax[k], c);
            }
        int best_axis = -1;
        double best_plane = 0, best_cost = INF;
        for (int k = 0; k < 3; ++k) {
            if (!(cmax[k] > cmin[k])) continue;
            for (int cnd = 1; cnd <= 3; ++cnd) {
                double plane = cmin[k] + (cmax[k] - cmin[k]) * cnd / 4.0;
                Box L, R;
                for (int a = 0; a < 3; ++a) { L.lo[a] = R.lo[a] = INF; L.hi[a] = R.hi[a] = -INF; }
                int nl = 0, nr = 0;
                for (int i = lo; i < hi; ++i) {
                    int id = ids_[size_t(i)];
                    const Box& b = (*boxes_)[size_t(id)];
                    Box& t = centre(id, k) < plane ? (++nl, L) : (++nr, R);
                    for (int a = 0; a < 3; ++a) { t.lo[a] = std::min(t.lo[a], b.lo[a]); t.hi[a] = std::max(t.hi[a], b.hi[a]); }
                }
                if (nl == 0 || nr == 0) continue;
                double cost = nl * area(L) + nr * area(R);
                if (cost < best_cost) { best_cost = cost; best_axis = k; best_plane = plane; }
            }
        }
        if (best_axis < 0) {
            // median fallback; the BIH takes the axis of widest centre spread
            last_axis = 0;
            for (int k = 1; k < 3; ++k)
                if (cmax[k] - cmin[k] > cmax[last_axis] - cmin[last_axis]) last_axis = k;
            return lo + n / 2;
        }
        last_axis = best_axis;
        auto it = std::partition(ids_.begin() + lo, ids_.begin() + hi,
                                 [&](int id) { return centre(id, best_axis) < best_plane; });
        return int(it - ids_.begin());
    }
    int last_axis = 0;

  public:
    // Bounding interval hierarchy over the same cells (Sec. 4.3): the same
    // SAH partition of the box centres; each node keeps the split axis, the
    // largest upper bound of the left set's boxes and the smallest lower
    // bound of the right set's along it (FP32, rounded outward).  Returns
    // the root reference.
    std::vector<BihNode> bih;
    int bih_depth = 0;
    int build_bih(std::vector<int>& cells, const std::vector<Box>& boxes) {
        ids_ = cells;
        boxes_ = &boxes;
        return emit_bih(0, int(ids_.size()), 0);
    }

  private:
    int emit_bih(int lo, int hi, int depth) {
        bih_depth = std::max(bih_depth, depth);
        if (hi - lo <= BVH_LEAF_MAX) {
            const int first = int(leaf_cells.size());
            for (int i = lo; i < hi; ++i) leaf_cells.push_back(ids_[size_t(i)]);
            return -1 - ((first << 4) | (hi - lo));
        }
        const int self = int(bih.size());
        bih.push_back(BihNode{});
        const int mid = depth > 24 ? lo + (hi - lo) / 2 : split(lo, hi);
        int axis = last_axis;
        if (depth > 24) {
            // median split below depth 24: axis of the widest centre spread
            double cmin[3] = {INF, INF, INF}, cmax[3] = {-INF, -INF, -INF};
            for (int i = lo; i < hi; ++i)
                for (int k = 0; k < 3; ++k) {
                    const double c = centre(ids_[size_t(i)], k);
                    cmin[k] = std::min(cmin[k], c); cmax[k] = std::max(cmax[k], c);
                }
            axis = 0;
            for (int k = 1; k < 3; ++k)
                if (cmax[k] - cmin[k] > cmax[axis] - cmin[axis]) axis = k;
        }
        const Box b0 = bound(lo, mid), b1 = bound(mid, hi);
        const int r0 = emit_bih(lo, mid, depth + 1);
        const int r1 = emit_bih(mid, hi, depth + 1);
        BihNode& nd = bih[size_t(self)];
        nd.clip_l = f_up(b0.hi[axis]);
        nd.clip_r = f_down(b1.lo[axis]);
        nd.ref0 = r0;
        nd.ref1_axis = r1 * 4 + axis;
        return self;
    }
  public:
    // SAH splits; below depth 24 the median, so the depth stays below
    // 24 + log2(cells) (the device walk's stack holds BVH_STACK entries).
    int emit(int lo, int hi, int depth) {
        max_depth = std::max(max_depth, depth);
        if (hi - lo <= BVH_LEAF_MAX) {
            const int first = int(leaf_cells.size());
            for (int i = lo; i < hi; ++i) leaf_cells.push_back(ids_[size_t(i)]);
            return -1 - ((first << 4) | (hi - lo));
        }
        const int self = int(nodes.size());
        nodes.push_back(BvhNode{});
        const int mid = depth > 24 ? lo + (hi - lo) / 2 : split(lo, hi);
        const Box b0 = bound(lo, mid), b1 = bound(mid, hi);
        const int r0 = emit(lo, mid, depth + 1);
        const int r1 = emit(mid, hi, depth + 1);
        BvhNode& nd = nodes[size_t(self)];
        for (int k = 0; k < 3; ++k) {
            nd.lo0[k] = f_down(b0.lo[k]); nd.hi0[k] = f_up(b0.hi[k]);
            nd.lo1[k] = f_down(b1.lo[k]); nd.hi1[k] = f_up(b1.hi[k]);
        }
        nd.ref0 = r0;
        nd.ref1 = r1;
        nd.pad0 = nd.pad1 = 0;
        return self;
    }
};

// Host validation of the built search structures (the tracking kernels read
// them without bounds checks): every cell of a universe sits in exactly one
// leaf of its BVH and of its BIH, a leaf holds only that universe's cells,
// every BVH node box on the way to a leaf contains the leaf's cell boxes, and
// every BIH clip plane on the way bounds them on its side.  A failure is a
// builder defect, reported as TRK_E_DESC before anything is copied to the
// device.
int validate_hierarchy(const BvhBuilder& bvh, int first_cell, int ncells, int bvh_root, int bih_root,
                       const std::vector<Box>& boxes, int u) {
    struct Item { int ref; std::vector<int> path; };   // path: node index * 2 + child side
    for (int kind = 0; kind < 2; ++kind) {
        const int root = kind == 0 ? bvh_root : bih_root;
        if (root == -1) continue;
        std::vector<int> seen(size_t(ncells), 0);
        std::vector<Item> stack;
        stack.push_back(Item{root, {}});
        while (!stack.empty()) {
            Item it = std::move(stack.back());
            stack.pop_back();
            if (it.ref >= 0) {
                if (kind == 0 && size_t(it.ref) >= bvh.nodes.size()) return set_error(TRK_E_DESC, "universe %d: BVH node %d out of range", u, it.ref);
                if (kind == 1 && size_t(it.ref) >= bvh.bih.size()) return set_error(TRK_E_DESC, "universe %d: BIH node %d out of range", u, it.ref);
                if (it.path.size() > size_t(BVH_STACK)) return set_error(TRK_E_DESC, "universe %d: hierarchy deeper than %d", u, BVH_STACK);
                const int r0 = kind == 0 ? bvh.nodes[size_t(it.ref)].ref0 : bvh.bih[size_t(it.ref)].ref0;
                const int r1 = kind == 0 ? bvh.nodes[size_t(it.ref)].ref1 : (bvh.bih[size_t(it.ref)].ref1_axis >> 2);
                for (int side = 0; side < 2; ++side) {
                    Item ch{side == 0 ? r0 : r1, it.path};
                    ch.path.push_back(it.ref * 2 + side);
                    stack.push_back(std::move(ch));
                }
                continue;
            }
            const int leaf = -1 - it.ref, first = leaf >> 4, cnt = leaf & 15;
            if (first < 0 || size_t(first) + size_t(cnt) > bvh.leaf_cells.size())
                return set_error(TRK_E_DESC, "universe %d: leaf range out of bounds", u);
            for (int k = 0; k < cnt; ++k) {
                const int c = bvh.leaf_cells[size_t(first + k)];
                if (c < first_cell || c >= first_cell + ncells)
                    return set_error(TRK_E_DESC, "universe %d: a leaf holds cell %d of another universe", u, c);
                seen[size_t(c - first_cell)]++;
                const Box& b = boxes[size_t(c)];
                for (int pe : it.path) {
                    const int nd = pe >> 1, side = pe & 1;
                    bool ok = true;
                    if (kind == 0) {
                        const BvhNode& N = bvh.nodes[size_t(nd)];
                        const float* lo = side == 0 ? N.lo0 : N.lo1;
                        const float* hi = side == 0 ? N.hi0 : N.hi1;
                        for (int a = 0; a < 3; ++a) ok = ok && double(lo[a]) <= b.lo[a] && double(hi[a]) >= b.hi[a];
                    } else {
                        const BihNode& N = bvh.bih[size_t(nd)];
                        const int axis = N.ref1_axis & 3;
                        ok = side == 0 ? double(N.clip_l) >= b.hi[axis] : double(N.clip_r) <= b.lo[axis];
                    }
                    if (!ok)
                        return set_error(TRK_E_DESC, "universe %d: %s node %d does not bound cell %d", u,
                                         kind == 0 ? "BVH" : "BIH", nd, c);
                }
            }
        }
        for (int i = 0; i < ncells; ++i)
            if (seen[size_t(i)] != 1)
                return set_error(TRK_E_DESC, "universe %d: cell %d appears %d times in its %s", u, first_cell + i,
                                 seen[size_t(i)], kind == 0 ? "BVH" : "BIH");
    }
    return TRK_OK;
}

// Order key of a double (see okey_bits): integer comparisons of keys agree
// with IEEE comparisons of the values, -0 equal to +0.
long long okey(double v) {
    long long b;
    std::memcpy(&b, &v, 8);
    return okey_bits(b);
}

// ---------------------------------------------------------------------------
// Flattening
// ---------------------------------------------------------------------------
struct Layout {
    size_t total = 0;
    size_t put(size_t bytes) {
        size_t off = (total + 255) & ~size_t(255);
        total = off + bytes;
        return off;
    }
};

template <class T>
void copy_into(std::vector<unsigned char>& img, size_t off, const std::vector<T>& v) {
    if (!v.empty()) std::memcpy(img.data() + off, v.data(), v.size() * sizeof(T));
}

struct Built {
    std::vector<unsigned char> image;
    size_t offs[48] = {};
    HGeom G;
    int n_nodes = 0;
};

int build_host(const char* json, size_t len, Built& B) {
    HGeom& G = B.G;
    int st = parse(json, len, G);
    if (st != TRK_OK) return st;
    std::vector<int> height(G.univ.size(), 0);
    std::vector<char> busy(G.univ.size(), 0);
    st = count_instances(G, G.root, height, busy);
    if (st != TRK_OK) return st;
    // every universe must be nested below the root: the flattening below
    // places, boxes and numbers each one through its parents
    for (size_t u = 0; u < G.univ.size(); ++u)
        if (G.univ[u].ninst < 0) return set_error(TRK_E_DESC, "universe %zu is not reachable from the root", u);
    G.depth = height[size_t(G.root)] + 1;
    if (G.depth > MAXL)
        return set_error(TRK_E_UNSUPPORTED, "nesting depth %d exceeds the compiled maximum %d", G.depth, MAXL);
    for (auto& s : G.surf)
        if (s.type == S_P && std::fabs(s.c[0]) + std::fabs(s.c[1]) + std::fabs(s.c[2]) == 0)
            return set_error(TRK_E_DESC, "plane with zero normal");
    // rect view: one lattice record per rect universe; CSG view: pseudo-arrays
    const int nu = int(G.univ.size());
    std::vector<int> lat_of(size_t(nu), -1);
    int nlat = 0;
    int nhex = 0;
    for (int u = 0; u < nu; ++u) {
        if (G.univ[size_t(u)].type == UT_RECT) lat_of[size_t(u)] = nlat++;
        else if (G.univ[size_t(u)].type == UT_HEX) lat_of[size_t(u)] = -2 - nhex++;
    }
    for (int u = 0; u < nu; ++u) {
        HUniv& U = G.univ[size_t(u)];
        if (U.type == UT_HEX && u == G.root && U.bc[0] == BC_REFLECT)
            return set_error(TRK_E_UNSUPPORTED, "reflecting hex array faces are not supported");
        if (U.type != UT_CSG) make_pseudo_array(G, u);
        U.lat = lat_of[size_t(u)];
    }
    compute_boxes(G);

    // global cell numbering and BVHs
    std::vector<Box> boxes;
    int ncell = 0;
    for (auto& U : G.univ) {
        U.first_cell = ncell;
        for (auto& c : U.cells) {
            Box b;
            for (int k = 0; k < 3; ++k) { b.lo[k] = c.box[k]; b.hi[k] = c.box[3 + k]; }
            boxes.push_back(b);
            ++ncell;
        }
    }
    BvhBuilder bvh;
    for (auto& U : G.univ) {
        if (int(U.cells.size()) <= LINEAR_MAX) { U.bvh = -1; continue; }
        std::vector<int> ids;
        for (int i = 0; i < int(U.cells.size()); ++i) ids.push_back(U.first_cell + i);
        for (int k = 0; k < 3; ++k) {
            double lo = INF, hi = -INF;
            for (int id : ids) {
                if (std::isfinite(boxes[size_t(id)].lo[k])) lo = std::min(lo, boxes[size_t(id)].lo[k]);
                if (std::isfinite(boxes[size_t(id)].hi[k])) hi = std::max(hi, boxes[size_t(id)].hi[k]);
            }
            if (!(hi > lo)) { lo = -1.0; hi = 1.0; }
            double m = hi - lo;
            bvh.proxy.lo[k] = lo - m;
            bvh.proxy.hi[k] = hi + m;
        }
        U.bvh = bvh.build(ids, boxes);
        if (U.bvh < 0) U.bvh = -1;   // a single leaf: the linear scan does the same
        if (U.bvh >= 0) {
            std::vector<int> ids2;
            for (int i = 0; i < int(U.cells.size()); ++i) ids2.push_back(U.first_cell + i);
            U.bih = bvh.build_bih(ids2, boxes);
        }
    }
    if (bvh.bih_depth >= BVH_STACK) return set_error(TRK_E_DESC, "BIH depth %d exceeds %d", bvh.bih_depth, BVH_STACK);
    if (bvh.max_depth >= BVH_STACK) return set_error(TRK_E_DESC, "BVH depth %d exceeds %d", bvh.max_depth, BVH_STACK);
    for (size_t u = 0; u < G.univ.size(); ++u) {
        const HUniv& U = G.univ[u];
        if (U.bvh < 0) continue;
        st = validate_hierarchy(bvh, U.first_cell, int(U.cells.size()), U.bvh, U.bih, boxes, int(u));
        if (st != TRK_OK) return st;
    }
    B.n_nodes = int(bvh.nodes.size());

    // SoA arrays
    std::vector<int> s_info;
    std::vector<double> s_coef;
    for (auto& s : G.surf) {
        s_info.push_back(s.type | (s.bc << 4) | ((s.rparam + 1) << 8) | (s.pscale ? (1 << 12) : 0));
        s_coef.push_back(s.c[0]);
        s_coef.push_back(s.c[1]);
        s_coef.push_back(s.c[2]);
        s_coef.push_back(s.type == S_CZ ? s.c[2] * s.c[2] : s.c[3]);
    }
    std::vector<long long> s_key;
    for (auto& s : G.surf) s_key.push_back(s.type <= S_PZ ? okey(s.c[0]) : 0);
    std::vector<float4> s_coeff;
    for (auto& s : G.surf) {
        if (s.type == S_CZ) s_coeff.push_back(make_float4(float(s.c[0]), float(s.c[1]), float(s.c[2] * s.c[2]), float(s.c[2])));
        else s_coeff.push_back(make_float4(float(s.c[0]), float(s.c[1]), float(s.c[2]), float(s.c[3])));
    }
    std::vector<float> c_slabf;
    std::vector<int2> c_range, cs_adj;
    std::vector<int4> c_slab0, c_slab1, c_slabs;
    std::vector<longlong2> c_slabk;
    std::vector<int> cs, c_fill, c_off, c_fcls, rest_e;
    std::vector<int2> c_rest;
    std::vector<int4> c_pair;
    std::vector<double> c_tr;
    std::vector<int4> u_info;
    for (auto& U : G.univ) {
        // face adjacency: cells of this universe holding the same surface with
        // the opposite sense whose boxes touch the cell's box
        std::map<int, std::vector<std::pair<int, int>>> by_surf;
        for (int ci = 0; ci < int(U.cells.size()); ++ci)
            for (size_t k = 0; k < U.cells[size_t(ci)].surf.size(); ++k)
                by_surf[U.cells[size_t(ci)].surf[k]].push_back({ci, U.cells[size_t(ci)].sense[k]});
        // boxes overlap; across an axis plane the overlap must have positive
        // area in the plane (cells that only share an edge are not neighbours)
        auto overlap = [](const HCell& a, const HCell& b, int axis) {
            for (int k = 0; k < 3; ++k) {
                const double lo = std::max(a.box[k], b.box[k]), hi = std::min(a.box[3 + k], b.box[3 + k]);
                if (lo > hi) return false;
                if (k != axis && axis >= 0 && std::isfinite(lo) && std::isfinite(hi) &&
                    hi - lo <= 1e-6 * std::max(1.0, std::max(std::fabs(lo), std::fabs(hi))))
                    return false;
            }
            return true;
        };
        for (int ci = 0; ci < int(U.cells.size()); ++ci) {
            const HCell& c = U.cells[size_t(ci)];
            c_range.push_back(make_int2(int(cs.size()), int(c.surf.size())));
            for (size_t i = 0; i < c.surf.size(); ++i) {
                const int type = G.surf[size_t(c.surf[i])].type;
                cs.push_back((c.surf[i] << 4) | (type << 1) | (c.sense[i] > 0 ? 1 : 0));
                std::vector<int> cand;
                const int axis = type <= S_PZ ? type : -1;
                for (auto& pr : by_surf[c.surf[i]])
                    if (pr.first != ci && pr.second == -c.sense[i] && overlap(c, U.cells[size_t(pr.first)], axis))
                        cand.push_back(U.first_cell + pr.first);
                if (cand.size() > 2) cs_adj.push_back(make_int2(-2, -2));
                else cs_adj.push_back(make_int2(cand.size() > 0 ? cand[0] : -1, cand.size() > 1 ? cand[1] : -1));
            }
            // slab view: at most one lower and one upper axis plane per
            // dimension; the other surfaces (cylinders, general planes) are
            // listed as the cell's remaining entries
            int slab[6] = {-1, -1, -1, -1, -1, -1};
            bool fits = true;
            const int first_entry = c_range.back().x;
            std::vector<int> rest;
            for (size_t i = 0; i < c.surf.size(); ++i) {
                const int type = G.surf[size_t(c.surf[i])].type;
                if (type > S_PZ) { rest.push_back(first_entry + int(i)); continue; }
                const int slot = 2 * type + (c.sense[i] > 0 ? 0 : 1);
                if (slab[slot] >= 0) { fits = false; break; }
                slab[slot] = first_entry + int(i);
            }
            // plane pairs: general planes with one normal (exactly equal
            // coefficients), at most one "+" and one "-" entry each (the two
            // faces of a hex element across one face family); up to three
            int pair[6] = {-1, -1, -1, -1, -1, -1};
            int npair = 0;
            if (fits) {
                std::vector<int> keep;
                for (int e : rest) {
                    const HSurf& sf = G.surf[size_t(c.surf[size_t(e - first_entry)])];
                    const int sense = c.sense[size_t(e - first_entry)];
                    if (sf.type != S_P) { keep.push_back(e); continue; }
                    int f = 0;
                    for (; f < npair; ++f) {
                        const int e0 = pair[2 * f] >= 0 ? pair[2 * f] : pair[2 * f + 1];
                        const HSurf& s0 = G.surf[size_t(c.surf[size_t(e0 - first_entry)])];
                        if (s0.c[0] == sf.c[0] && s0.c[1] == sf.c[1] && s0.c[2] == sf.c[2]) break;
                    }
                    const int slot = sense > 0 ? 0 : 1;
                    if (f < npair && pair[2 * f + slot] < 0) { pair[2 * f + slot] = e; continue; }
                    if (f == npair && npair < 3) { pair[2 * f + slot] = e; ++npair; continue; }
                    keep.push_back(e);
                }
                rest.swap(keep);
            }
            // a cell with neither axis planes nor plane pairs (a pin cell
            // bounded by cylinders) keeps the plain entry loop
            bool any_axis = false;
            for (int k = 0; k < 6; ++k) any_axis |= slab[k] >= 0;
            if (!any_axis && npair == 0) fits = false;
            if (!fits) {
                for (int k = 0; k < 6; ++k) slab[k] = pair[k] = -1;
                npair = 0;
                rest.clear();
                c_rest.push_back(make_int2(int(rest_e.size()), 0));
            } else {
                c_range.back().y |= CS_SLAB_FLAG;
                if (npair > 0) c_range.back().y |= CS_PAIR_FLAG;
                c_rest.push_back(make_int2(int(rest_e.size()), int(rest.size())));
                rest_e.insert(rest_e.end(), rest.begin(), rest.end());
            }
            c_pair.push_back(make_int4(pair[0], pair[1], pair[2], pair[3]));
            c_pair.push_back(make_int4(pair[4], pair[5], -1, -1));
            for (int k = 0; k < 6; ++k) {
                const int e = slab[k];
                c_slabf.push_back(e >= 0 ? float(G.surf[size_t(c.surf[size_t(e - first_entry)])].c[0] - c.tr[k / 2]) : 0.f);
            }
            c_slab0.push_back(make_int4(slab[0], slab[1], slab[2], slab[3]));
            c_slab1.push_back(make_int4(slab[4], slab[5], 0, 0));
            int sid6[6];
            for (int k = 0; k < 6; ++k) sid6[k] = slab[k] >= 0 ? c.surf[size_t(slab[k] - first_entry)] : -1;
            for (int d = 0; d < 3; ++d) {
                const int lo = sid6[2 * d], hi = sid6[2 * d + 1];
                longlong2 kk;
                kk.x = lo >= 0 ? okey(G.surf[size_t(lo)].c[0]) : std::numeric_limits<long long>::min();
                kk.y = hi >= 0 ? okey(G.surf[size_t(hi)].c[0]) : std::numeric_limits<long long>::max();
                c_slabk.push_back(kk);
            }
            c_slabs.push_back(make_int4(sid6[0], sid6[1], sid6[2], sid6[3]));
            c_slabs.push_back(make_int4(sid6[4], sid6[5], -1, -1));
            {
                int curved = 0, general = 0, cyl_side = 0;
                for (size_t i = 0; i < c.surf.size(); ++i) {
                    const int type = G.surf[size_t(c.surf[i])].type;
                    if (type == S_CZ) { ++curved; cyl_side = c.sense[i]; }
                    else if (type == S_P) ++general;
                }
                int cls = 3;
                if (general == 0 && curved == 0) cls = 0;
                else if (general == 0 && curved == 1) cls = cyl_side < 0 ? 1 : 2;
                c_fcls.push_back(cls);
            }
            c_fill.push_back(c.fill);
            c_off.push_back(int(c.off));
            for (int d = 0; d < 3; ++d) c_tr.push_back(c.tr[d]);
        }
        u_info.push_back(make_int4(U.first_cell, int(U.cells.size()), U.bvh, U.lat));
    }
    std::vector<int4> l_dim, l_off;
    std::vector<double> l_grid, l_ctr;
    std::vector<long long> l_gkey;
    std::vector<float> l_lof, l_hif;
    std::vector<int> l_fill, l_eoff, l_pscale;
    for (auto& U : G.univ) {
        if (U.type != UT_RECT) continue;
        int4 dm, of;
        int n[3];
        int go[3];
        for (int d = 0; d < 3; ++d) {
            n[d] = int(U.grid[d].size()) - 1;
            go[d] = int(l_grid.size());
            for (double g : U.grid[d]) { l_grid.push_back(g); l_gkey.push_back(okey(g)); }
            for (int i = 0; i < n[d]; ++i) {
                const double c = (U.grid[d][size_t(i)] + U.grid[d][size_t(i) + 1]) * 0.5;
                l_ctr.push_back(c);
                l_lof.push_back(float(U.grid[d][size_t(i)] - c));
                l_hif.push_back(float(U.grid[d][size_t(i) + 1] - c));
            }
            l_ctr.push_back(0.0);   // keep l_ctr aligned with l_grid offsets
            l_lof.push_back(0.f);
            l_hif.push_back(0.f);
        }
        int bcp = 0;
        for (int k = 0; k < 6; ++k) bcp |= (U.bc[k] & 3) << (2 * k);
        dm = make_int4(n[0], n[1], n[2], bcp);
        of = make_int4(go[0], go[1], go[2], int(l_fill.size()));
        for (size_t e = 0; e < U.fill.size(); ++e) { l_fill.push_back(U.fill[e]); l_eoff.push_back(int(U.eoff[e])); }
        l_dim.push_back(dm);
        l_off.push_back(of);
        l_pscale.push_back(U.pscale);
    }
    if (l_dim.empty()) { l_dim.push_back(make_int4(0, 0, 0, 0)); l_off.push_back(make_int4(0, 0, 0, 0)); l_pscale.push_back(0); }
    // hex lattices (array tracker): inverse lattice matrix and row starts
    std::vector<HexInfo> hx;
    std::vector<int> hx_row;
    for (auto& U : G.univ) {
        if (U.type != UT_HEX) continue;
        HexInfo h;
        std::memset(&h, 0, sizeof h);
        const double det = U.a1[0] * U.a2[1] - U.a2[0] * U.a1[1];
        h.i00 = U.a2[1] / det; h.i01 = -U.a2[0] / det;
        h.i10 = -U.a1[1] / det; h.i11 = U.a1[0] / det;
        h.rings = U.rings;
        h.first_cell = U.first_cell;
        h.row = int(hx_row.size());
        const int R = U.rings;
        int e = 0;
        for (int r = -R; r <= R; ++r) {
            hx_row.push_back(e);
            e += std::min(R, R - r) - std::max(-R, -R - r) + 1;
        }
        hx.push_back(h);
    }
    if (hx.empty()) { HexInfo h; std::memset(&h, 0, sizeof h); hx.push_back(h); }
    if (hx_row.empty()) hx_row.push_back(0);
    if (l_grid.empty()) { l_grid.push_back(0); l_ctr.push_back(0); l_gkey.push_back(0); l_lof.push_back(0); l_hif.push_back(0); }
    if (c_slabf.empty()) c_slabf.push_back(0);
    if (l_fill.empty()) { l_fill.push_back(0); l_eoff.push_back(0); }
    std::vector<BvhNode> nodes = bvh.nodes;
    std::vector<int> leaf = bvh.leaf_cells;
    if (nodes.empty()) nodes.push_back(BvhNode{});
    if (leaf.empty()) leaf.push_back(0);
    if (cs.empty()) { cs.push_back(0); cs_adj.push_back(make_int2(-1, -1)); }

    Layout L;
    size_t* o = B.offs;
    o[0] = L.put(s_info.size() * 4);
    o[1] = L.put(s_coef.size() * sizeof(double));
    o[2] = L.put(c_range.size() * sizeof(int2));
    o[3] = L.put(cs.size() * 4);
    o[4] = L.put(c_fill.size() * 4);
    o[5] = L.put(c_tr.size() * 8);
    o[6] = L.put(c_off.size() * 4);
    o[7] = L.put(u_info.size() * sizeof(int4));
    o[8] = L.put(l_dim.size() * sizeof(int4));
    o[9] = L.put(l_off.size() * sizeof(int4));
    o[10] = L.put(l_grid.size() * 8);
    o[11] = L.put(l_ctr.size() * 8);
    o[12] = L.put(l_fill.size() * 4);
    o[13] = L.put(l_eoff.size() * 4);
    o[14] = L.put(l_pscale.size() * 4);
    o[15] = L.put(nodes.size() * sizeof(BvhNode));
    o[16] = L.put(leaf.size() * 4);
    o[17] = L.put(G.sigma.size() * 8);
    o[39] = L.put(G.nu.size() * 8);
    std::vector<double> rsigma;
    for (double v : G.sigma) rsigma.push_back(v > 0.0 ? 1.0 / v : 0.0);
    o[41] = L.put(rsigma.size() * 8);
    o[18] = L.put(s_key.size() * 8);
    o[19] = L.put(cs_adj.size() * sizeof(int2));
    o[20] = L.put(l_gkey.size() * 8);
    o[21] = L.put(c_slab0.size() * sizeof(int4));
    o[22] = L.put(c_slab1.size() * sizeof(int4));
    o[23] = L.put(s_coeff.size() * sizeof(float4));
    o[24] = L.put(l_lof.size() * 4);
    o[25] = L.put(l_hif.size() * 4);
    o[26] = L.put(c_slabf.size() * 4);
    if (c_slabk.empty()) { c_slabk.push_back(longlong2{0, 0}); c_slabs.push_back(make_int4(-1, -1, -1, -1)); }
    o[27] = L.put(c_slabk.size() * sizeof(longlong2));
    o[28] = L.put(c_slabs.size() * sizeof(int4));
    if (c_fcls.empty()) c_fcls.push_back(0);
    o[29] = L.put(c_fcls.size() * 4);
    if (c_rest.empty()) c_rest.push_back(make_int2(0, 0));
    if (rest_e.empty()) rest_e.push_back(0);
    o[30] = L.put(c_rest.size() * sizeof(int2));
    o[31] = L.put(rest_e.size() * 4);
    o[32] = L.put(hx.size() * sizeof(HexInfo));
    o[33] = L.put(hx_row.size() * 4);
    if (c_pair.empty()) { c_pair.push_back(make_int4(-1, -1, -1, -1)); c_pair.push_back(make_int4(-1, -1, -1, -1)); }
    o[34] = L.put(c_pair.size() * sizeof(int4));
    std::vector<int> u_bih;
    for (auto& U : G.univ) u_bih.push_back(U.bih);
    std::vector<BihNode> bihn = bvh.bih;
    if (bihn.empty()) bihn.push_back(BihNode{});
    o[37] = L.put(u_bih.size() * 4);
    o[38] = L.put(bihn.size() * sizeof(BihNode));
    std::vector<double> m_grid;
    std::vector<long long> m_key;
    for (int d = 0; d < 3; ++d)
        for (double v : G.mesh[d]) { m_grid.push_back(v); m_key.push_back(okey(v)); }
    if (m_grid.empty()) { m_grid.push_back(0.0); m_key.push_back(0); }
    o[35] = L.put(m_grid.size() * 8);
    o[36] = L.put(m_key.size() * 8);
    o[40] = L.put(TRK_DP_BYTES);        // DP tracker objects, built on the device
    B.image.assign(L.total, 0);
    copy_into(B.image, o[0], s_info);
    copy_into(B.image, o[1], s_coef);
    copy_into(B.image, o[2], c_range);
    copy_into(B.image, o[3], cs);
    copy_into(B.image, o[4], c_fill);
    copy_into(B.image, o[5], c_tr);
    copy_into(B.image, o[6], c_off);
    copy_into(B.image, o[7], u_info);
    copy_into(B.image, o[8], l_dim);
    copy_into(B.image, o[9], l_off);
    copy_into(B.image, o[10], l_grid);
    copy_into(B.image, o[11], l_ctr);
    copy_into(B.image, o[12], l_fill);
    copy_into(B.image, o[13], l_eoff);
    copy_into(B.image, o[14], l_pscale);
    copy_into(B.image, o[15], nodes);
    copy_into(B.image, o[16], leaf);
    copy_into(B.image, o[17], G.sigma);
    copy_into(B.image, o[39], G.nu);
    copy_into(B.image, o[41], rsigma);
    copy_into(B.image, o[18], s_key);
    copy_into(B.image, o[19], cs_adj);
    copy_into(B.image, o[20], l_gkey);
    copy_into(B.image, o[21], c_slab0);
    copy_into(B.image, o[22], c_slab1);
    copy_into(B.image, o[23], s_coeff);
    copy_into(B.image, o[24], l_lof);
    copy_into(B.image, o[25], l_hif);
    copy_into(B.image, o[26], c_slabf);
    copy_into(B.image, o[27], c_slabk);
    copy_into(B.image, o[28], c_slabs);
    copy_into(B.image, o[29], c_fcls);
    copy_into(B.image, o[30], c_rest);
    copy_into(B.image, o[31], rest_e);
    copy_into(B.image, o[32], hx);
    copy_into(B.image, o[33], hx_row);
    copy_into(B.image, o[34], c_pair);
    copy_into(B.image, o[37], u_bih);
    copy_into(B.image, o[38], bihn);
    copy_into(B.image, o[35], m_grid);
    copy_into(B.image, o[36], m_key);
    return TRK_OK;
}

}  // namespace
}  // namespace trk

using namespace trk;

extern "C" {

const char* trk_last_error(void) { return t_err.c_str(); }

void trk_default_opts(trk_run_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->tracker = TRK_TRACKER_AUTO;
    o->mode = TRK_MODE_HISTORY;
    o->precision = TRK_FP64;
    o->seed = 1;
    o->max_segments = 1000000;
    o->p_absorb = 0.3;
    o->max_path = 0.0;
}

trk_status geometry_build(const char* json, size_t len, void* dev_buf, size_t* dev_bytes, void* stream,
                          trk_geom_t* out) {
    t_err.clear();
    if (!json || !dev_bytes) return trk_status(set_error(TRK_E_INVALID, "geometry_build: null json or dev_bytes"));
    Built B;
    int st = build_host(json, len, B);
    if (st != TRK_OK) return trk_status(st);
    size_t need = B.image.size();
    if (!dev_buf) { *dev_bytes = need; return TRK_OK; }
    if (!out) return trk_status(set_error(TRK_E_INVALID, "geometry_build: null out handle"));
    if (*dev_bytes < need) {
        size_t have = *dev_bytes;
        *dev_bytes = need;
        return trk_status(set_error(TRK_E_NOMEM, "geometry_build: buffer of %zu bytes, need %zu", have, need));
    }
    if ((reinterpret_cast<uintptr_t>(dev_buf) & 255) != 0)
        return trk_status(set_error(TRK_E_INVALID, "geometry_build: dev_buf must be 256-byte aligned"));
    cudaError_t ce = cudaMemcpyAsync(dev_buf, B.image.data(), need, cudaMemcpyHostToDevice,
                                     static_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "geometry_build: cudaMemcpyAsync: %s", cudaGetErrorString(ce)));
    ce = cudaError_t(dp_install(static_cast<unsigned char*>(dev_buf) + B.offs[40], stream));
    if (ce != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "geometry_build: DP trackers: %s", cudaGetErrorString(ce)));
    // the staging image is pageable host memory: wait for the copy before it goes away
    ce = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) return trk_status(set_error(TRK_E_CUDA, "geometry_build: %s", cudaGetErrorString(ce)));
    *dev_bytes = need;
    trk_geom* h = new trk_geom;
    unsigned char* base = static_cast<unsigned char*>(dev_buf);
    DevGeom& d = h->dg;
    const size_t* o = B.offs;
    d.s_info = reinterpret_cast<const int*>(base + o[0]);
    d.s_coef = reinterpret_cast<const double*>(base + o[1]);
    d.c_range = reinterpret_cast<const int2*>(base + o[2]);
    d.cs = reinterpret_cast<const int*>(base + o[3]);
    d.c_fill = reinterpret_cast<const int*>(base + o[4]);
    d.c_tr = reinterpret_cast<const double*>(base + o[5]);
    d.c_off = reinterpret_cast<const int*>(base + o[6]);
    d.dp = base + o[40];
    d.u_info = reinterpret_cast<const int4*>(base + o[7]);
    d.l_dim = reinterpret_cast<const int4*>(base + o[8]);
    d.l_off = reinterpret_cast<const int4*>(base + o[9]);
    d.l_grid = reinterpret_cast<const double*>(base + o[10]);
    d.l_ctr = reinterpret_cast<const double*>(base + o[11]);
    d.l_fill = reinterpret_cast<const int*>(base + o[12]);
    d.l_eoff = reinterpret_cast<const int*>(base + o[13]);
    d.l_pscale = reinterpret_cast<const int*>(base + o[14]);
    d.nodes = reinterpret_cast<const BvhNode*>(base + o[15]);
    d.leaf_cells = reinterpret_cast<const int*>(base + o[16]);
    d.sigma = reinterpret_cast<const double*>(base + o[17]);
    d.rsigma = reinterpret_cast<const double*>(base + o[41]);
    d.nu = reinterpret_cast<const double*>(base + o[39]);
    d.s_key = reinterpret_cast<const long long*>(base + o[18]);
    d.cs_adj = reinterpret_cast<const int2*>(base + o[19]);
    d.l_gkey = reinterpret_cast<const long long*>(base + o[20]);
    d.c_slab0 = reinterpret_cast<const int4*>(base + o[21]);
    d.c_slab1 = reinterpret_cast<const int4*>(base + o[22]);
    d.s_coeff = reinterpret_cast<const float4*>(base + o[23]);
    d.l_lof = reinterpret_cast<const float*>(base + o[24]);
    d.l_hif = reinterpret_cast<const float*>(base + o[25]);
    d.c_slabf = reinterpret_cast<const float*>(base + o[26]);
    d.c_slabk = reinterpret_cast<const longlong2*>(base + o[27]);
    d.c_slabs = reinterpret_cast<const int4*>(base + o[28]);
    d.c_fcls = reinterpret_cast<const int*>(base + o[29]);
    d.c_rest = reinterpret_cast<const int2*>(base + o[30]);
    d.rest_e = reinterpret_cast<const int*>(base + o[31]);
    d.hx = reinterpret_cast<const HexInfo*>(base + o[32]);
    d.hx_row = reinterpret_cast<const int*>(base + o[33]);
    d.c_pair = reinterpret_cast<const int4*>(base + o[34]);
    d.u_bih = reinterpret_cast<const int*>(base + o[37]);
    d.bih = reinterpret_cast<const BihNode*>(base + o[38]);
    d.accel = B.G.accel;
    d.m_grid = reinterpret_cast<const double*>(base + o[35]);
    d.m_key = reinterpret_cast<const long long*>(base + o[36]);
    {
        int go = 0;
        for (int k = 0; k < 3; ++k) {
            const std::vector<double>& mg = B.G.mesh[k];
            d.m_n[k] = mg.empty() ? 0 : int(mg.size()) - 1;
            d.m_go[k] = go;
            d.m_lo[k] = mg.empty() ? 0.0 : mg.front();
            d.m_inv[k] = mg.empty() ? 0.0 : double(d.m_n[k]) / (mg.back() - mg.front());
            go += int(mg.size());
        }
    }
    const HGeom& G = B.G;
    for (int k = 0; k < 3; ++k) { d.src_lo[k] = G.src[k]; d.src_hi[k] = G.src[3 + k]; }
    d.root = G.root;
    d.n_inst = int(G.univ[size_t(G.root)].ninst);
    d.n_mat = int(G.sigma.size());
    d.gid = G.gid;
    d.max_depth = G.depth;
    d.n_univ = int(G.univ.size());
    int nc = 0;
    for (auto& U : G.univ) nc += int(U.cells.size());
    d.n_cells = nc;
    d.n_surf = int(G.surf.size());
    d.rect_ok = G.rect_ok ? 1 : 0;
    h->bytes = need;
    h->n_inst = d.n_inst;
    h->n_mat = d.n_mat;
    h->depth = d.max_depth;
    h->rect_ok = d.rect_ok;
    for (auto& U : G.univ) h->has_hex |= U.type == UT_HEX ? 1 : 0;
    h->n_nodes = B.n_nodes;
    for (auto& U : G.univ)
        if (U.type == UT_RECT)
            for (int k = 0; k < 3; ++k) h->max_rect_dim = std::max(h->max_rect_dim, int(U.grid[k].size()) - 1);
    h->magic = TRK_GEOM_MAGIC;
    *out = h;
    return TRK_OK;
}

trk_status geometry_destroy(trk_geom_t g) {
    if (!g || g->magic != TRK_GEOM_MAGIC) return trk_status(set_error(TRK_E_INVALID, "geometry_destroy: invalid handle"));
    g->magic = 0;
    delete g;
    return TRK_OK;
}

trk_status geometry_info(trk_geom_t g, int64_t* n_instances, int32_t* n_materials, int32_t* max_depth,
                         int32_t* rect_ok) {
    if (!g || g->magic != TRK_GEOM_MAGIC) return trk_status(set_error(TRK_E_INVALID, "geometry_info: invalid handle"));
    if (n_instances) *n_instances = g->n_inst;
    if (n_materials) *n_materials = g->n_mat;
    if (max_depth) *max_depth = g->depth;
    if (rect_ok) *rect_ok = g->rect_ok;
    return TRK_OK;
}

trk_status geometry_mesh_bins(trk_geom_t g, int64_t* bins) {
    if (!g || g->magic != TRK_GEOM_MAGIC || !bins) return trk_status(set_error(TRK_E_INVALID, "geometry_mesh_bins: bad arguments"));
    *bins = (int64_t)g->dg.m_n[0] * g->dg.m_n[1] * g->dg.m_n[2];
    return TRK_OK;
}

}  // extern "C"
