/*
 * flops.cpp -- operation count of the oracle's VMS operators.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY, like the oracle it counts:
 * nothing in the product path links or calls it.  It gives the algorithmic
 * flop count per element that the benchmark divides by a kernel's time.
 *
 * How it counts.  fsi_oracle.c is compiled a second time as C++ with every
 * FP64 value replaced by a counting number (`cnum`): the value plus a value
 * number.  Each + - * / and sqrt that the oracle executes is one operation,
 * except
 *   - operations on constants only (shape functions at the Gauss points,
 *     the metric G, det J, C_I nu^2 G:G on the uniform grid, the chain
 *     factors): they do not depend on the element's data, so they are
 *     folded (hoisted out of the element loop);
 *   - x + 0, x - 0, 0 - x, x * 1, x * -1, x * 0 and x / 1, which need no
 *     arithmetic;
 *   - an operation already applied to the same operands (same value
 *     numbers) in the same pass: common subexpressions are counted once.
 * So the count is the number of distinct arithmetic operations in the
 * oracle's computation of one element, as written (sums over the 8 nodes at
 * each Gauss point, per test node contributions), with nothing reassociated
 * or factorised.  Inputs get unique value numbers; physical parameters are
 * generic values (rho = 1.3, mu = 0.02, dt = 1e-3), so no identity depends
 * on them; the configuration is the benchmark's (no s field, no body force).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <cmath>
#include <cstring>
#include <unordered_map>
#include <utility>

namespace count {

long long g_ops = 0;
long long g_next = 1;  // value numbers of data-derived values are >= 1

struct Key {
    int op;
    long long a, b;
    bool operator==(const Key &o) const { return op == o.op && a == o.a && b == o.b; }
};
struct KeyHash {
    size_t operator()(const Key &k) const
    {
        return std::hash<long long>()(k.a * 1000003LL ^ (k.b * 7919LL) ^ (long long)k.op);
    }
};
std::unordered_map<Key, std::pair<double, long long>, KeyHash> g_seen;

// Constants carry value number <= 0: 0 for the value 0 (also what memset and
// calloc leave), a negative number derived from the bits otherwise.
long long const_id(double v)
{
    if (v == 0.0) return 0;
    long long b;
    std::memcpy(&b, &v, sizeof b);
    return -1 - (long long)((unsigned long long)b % (1ULL << 61));
}

}  // namespace count

struct cnum {
    double v;
    long long id;
    cnum() = default;
    cnum(double x) : v(x), id(count::const_id(x)) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    explicit operator long long() const { return (long long)v; }
};

namespace count {

constexpr long long kNegBit = 1LL << 62;

inline bool is_const(const cnum &a) { return a.id <= 0; }
inline cnum make(double v, long long id)
{
    cnum c;
    c.v = v;
    c.id = id;
    return c;
}
inline cnum negate(const cnum &a) { return is_const(a) ? cnum(-a.v) : make(-a.v, a.id ^ kNegBit); }

// op: 0 add, 1 sub, 2 mul, 3 div, 4 sqrt
cnum apply(int op, const cnum &a, const cnum &b)
{
    double r = op == 0 ? a.v + b.v : op == 1 ? a.v - b.v : op == 2 ? a.v * b.v
             : op == 3 ? a.v / b.v : std::sqrt(a.v);
    if (is_const(a) && (op == 4 || is_const(b))) return cnum(r);
    if (op == 0) {
        if (is_const(a) && a.v == 0.0) return b;
        if (is_const(b) && b.v == 0.0) return a;
    } else if (op == 1) {
        if (is_const(b) && b.v == 0.0) return a;
        if (is_const(a) && a.v == 0.0) return negate(b);
    } else if (op == 2) {
        if ((is_const(a) && a.v == 0.0) || (is_const(b) && b.v == 0.0)) return cnum(0.0);
        if (is_const(a) && a.v == 1.0) return b;
        if (is_const(b) && b.v == 1.0) return a;
        if (is_const(a) && a.v == -1.0) return negate(b);
        if (is_const(b) && b.v == -1.0) return negate(a);
    } else if (op == 3) {
        if (is_const(b) && b.v == 1.0) return a;
    }
    long long x = a.id, y = op == 4 ? 0 : b.id;
    if ((op == 0 || op == 2) && x > y) std::swap(x, y);
    Key k{op, x, y};
    auto it = g_seen.find(k);
    if (it != g_seen.end()) return make(it->second.first, it->second.second);
    ++g_ops;
    const long long id = g_next++;
    g_seen[k] = {r, id};
    return make(r, id);
}

}  // namespace count

#define CNUM_OP(o, c)                                                                   \
    inline cnum operator o(cnum a, cnum b) { return count::apply(c, a, b); }            \
    inline cnum operator o(cnum a, double b) { return count::apply(c, a, cnum(b)); }    \
    inline cnum operator o(double a, cnum b) { return count::apply(c, cnum(a), b); }    \
    inline cnum operator o(cnum a, int b) { return count::apply(c, a, cnum((double)b)); } \
    inline cnum operator o(int a, cnum b) { return count::apply(c, cnum((double)a), b); } \
    inline cnum &operator o##=(cnum & a, cnum b)                                        \
    {                                                                                   \
        a = count::apply(c, a, b);                                                      \
        return a;                                                                       \
    }
CNUM_OP(+, 0)
CNUM_OP(-, 1)
CNUM_OP(*, 2)
CNUM_OP(/, 3)
#undef CNUM_OP
inline cnum operator-(cnum a) { return count::negate(a); }
#define CNUM_CMP(o)                                                      \
    inline bool operator o(cnum a, cnum b) { return a.v o b.v; }         \
    inline bool operator o(cnum a, double b) { return a.v o b; }         \
    inline bool operator o(double a, cnum b) { return a o b.v; }         \
    inline bool operator o(cnum a, int b) { return a.v o(double) b; }
CNUM_CMP(<)
CNUM_CMP(>)
CNUM_CMP(<=)
CNUM_CMP(>=)
CNUM_CMP(==)
CNUM_CMP(!=)
#undef CNUM_CMP
inline cnum sqrt(cnum a) { return count::apply(4, a, cnum(0.0)); }
inline cnum fabs(cnum a) { return count::make(std::fabs(a.v), a.id); }
inline cnum floor(cnum a) { return cnum(std::floor(a.v)); }
inline bool isnan(cnum a) { return std::isnan(a.v); }
inline bool isfinite(cnum a) { return std::isfinite(a.v); }

#define double cnum
#include "fsi_oracle.c"
#undef double

namespace {

struct Fields {
    long n;
    cnum *U, *A, *x, *R, *J;
};

Fields make_fields(const int N[3])
{
    Fields F;
    F.n = (long)(N[0] + 1) * (N[1] + 1) * (N[2] + 1);
    cnum **arrs[] = {&F.U, &F.A, &F.x, &F.R, &F.J};
    for (cnum **p : arrs) *p = (cnum *)calloc((size_t)F.n * 4, sizeof(cnum));
    for (long i = 0; i < 4 * F.n; ++i) {
        F.U[i] = count::make(0.1 + 1e-3 * (double)i, count::g_next++);
        F.A[i] = count::make(0.2 + 2e-3 * (double)i, count::g_next++);
        F.x[i] = count::make(0.3 + 3e-3 * (double)i, count::g_next++);
    }
    for (long i = 0; i < F.n; ++i) F.A[4 * i + 3] = cnum(1.0);  // no s field
    return F;
}

void free_fields(Fields &F)
{
    free(F.U);
    free(F.A);
    free(F.x);
    free(F.R);
    free(F.J);
}

}  // namespace

/* Operations per element of the oracle's residual (what = 0), Jacobian apply
 * (1) or of both at the same state (2: what they share is counted once), on
 * an N^3 grid of spacing 1/N.  Common subexpressions are merged within one
 * element's computation only (no sharing between elements, whose kernels
 * run independently).  parts[0..2] receive the shares of the Gauss-point
 * evaluation of the fields (eval_gp), of the weak form at the Gauss points
 * (gp_residual / gp_jacobian, with the per-test-node terms) and of the
 * assembly into nodes: 32 - 4 n / E additions per element and operator (a
 * node's first contribution needs none).  Returns the total per element.
 * driver != 0 instead counts one call of the oracle's own assembled
 * operators (or_residual / or_jacobian_apply) with one table for the whole
 * grid; on a single element (N = 1) the two counts must agree.            */
extern "C" double or_count_vms_flops(int N, int what, int driver, double parts[3])
{
    const int Ns[3] = {N, N, N};
    const cnum h[3] = {cnum(1.0 / N), cnum(1.0 / N), cnum(1.0 / N)};
    const double rho = 1.3, mu = 0.02, dt = 1e-3, rho_inf = 0.5;
    const double am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf), af = 1.0 / (1.0 + rho_inf);
    const double gam = 0.5 + am - af;
    const cnum phys[5] = {cnum(rho), cnum(mu), cnum(4.0 / (dt * dt)), cnum(36.0), cnum(0.0)};
    const cnum c_a(am), c_v(af * gam * dt);
    const bool res = what == 0 || what == 2, jac = what == 1 || what == 2;
    Fields F = make_fields(Ns);
    const int64_t E = (int64_t)N * N * N;
    double total = 0.0;
    if (driver) {
        count::g_seen.clear();
        count::g_ops = 0;
        if (res) or_residual(Ns, h, phys, F.U, F.A, NULL, 1, F.R, 1);
        if (jac) or_jacobian_apply(Ns, h, phys, F.U, F.A, NULL, F.x, c_a, c_v, F.J, 1);
        total = (double)count::g_ops / (double)E;
        if (parts) parts[0] = parts[1] = parts[2] = 0.0;
    } else {
        or_phys ph = unpack_phys(phys);
        long long ev = 0, wf = 0;
        for (int64_t e = 0; e < E; ++e) {
            count::g_seen.clear();
            const int ex = (int)(e % N), ey = (int)((e / N) % N), ez = (int)(e / ((int64_t)N * N));
            cnum xe[8][4], Re[8][4], Je[8][4];
            for (int a = 0; a < 8; ++a)
                for (int c = 0; c < 4; ++c) xe[a][c] = F.x[4 * elem_node(Ns, ex, ey, ez, a) + c];
            memset(Re, 0, sizeof Re);
            memset(Je, 0, sizeof Je);
            for (int g = 0; g < 8; ++g) {
                gp_state st;
                const long long t0 = count::g_ops;
                eval_gp(Ns, h, NULL, ex, ey, ez, g, F.U, F.A, NULL, ph.has_s, &st);
                const long long t1 = count::g_ops;
                if (res) gp_residual(&st, &ph, 8, st.detJ, 1, Re);
                if (jac) gp_jacobian(&st, &ph, 8, st.detJ, xe, c_a, c_v, Je);
                ev += t1 - t0;
                wf += count::g_ops - t1;
            }
        }
        const double asm_ = (res + jac) * (32.0 * (double)E - 4.0 * (double)F.n) / (double)E;
        total = ((double)ev + (double)wf) / (double)E + asm_;
        if (parts) {
            parts[0] = (double)ev / (double)E;
            parts[1] = (double)wf / (double)E;
            parts[2] = asm_;
        }
    }
    free_fields(F);
    return total;
}
