// amg.cu -- pressure block of the Schur-complement block preconditioner on a
// tetrahedral mesh, and on a structured grid that asks for it (Sec. 2.4
// solves the reduced system with block preconditioners built from its
// sub-matrices).  The approximation is the one of the structured grid: the
// pressure Schur complement acts like sigma (K + kappa M), K and M now the
// stiffness and mass matrices of the pressure space as assembled from the
// elements (P1 on tetrahedra; Q1 on the hexahedra of the grid, through its
// mapped node coordinates when it has them, 2x2x2 Gauss points -- exact on
// affine maps; on a trilinear map K still passes the linear patch test and
// M integrates volume and first moments exactly), kappa = (pi / (2 L))^2 with L the
// largest extent of the mesh's bounding box.  Eliminated nodes (boundary nodes where
// the velocity is free, and nodes with a Dirichlet pressure) keep only their
// diagonal entry and drop out of every other row.  With no grid hierarchy,
// the inverse is one V-cycle of smoothed-aggregation algebraic multigrid
// (Vanek, Mandel and Brezina, Computing 56, 1996), set up on the host in
// FP64 once per elimination set:
//
//   strength    j is a strong neighbour of i if |a_ij| >= theta sqrt(a_ii a_jj),
//               theta = 0.08 on tetrahedra, 0.02 on hexahedra (the Q1
//               stiffness of a near-cubic element couples face neighbours by
//               ~0 and edge and corner neighbours by 1/16 and 1/32 of the
//               diagonal: 0.02 keeps all 26 neighbours strong);
//   aggregates  three greedy passes in node order: a node whose strong
//               neighbours are all free starts an aggregate with them; a free
//               node joins the first-pass aggregate of its strongest
//               neighbour; the rest form aggregates with their free strong
//               neighbours; nodes without strong neighbours (the eliminated
//               ones) join none;
//   transfer    P = (I - omega D^-1 A) P0, P0 the 0/1 aggregate indicator,
//               omega = 4 / (3 rho), rho the spectral radius of D^-1 A
//               (power iteration on D^-1/2 A D^-1/2, capped by Gershgorin);
//               restriction R = P^T; coarse operator R A P (Galerkin);
//   levels      until a level has <= 600 unknowns, coarsens by less than
//               a factor 1.25, or 16 levels;
//   smoother    Chebyshev semi-iteration of degree 2 on D^-1 A over
//               [hi/10, hi], hi = 1.1 rho (pre- and post-smoothing);
//   coarsest    a dense inverse (FP64 host Gauss-Jordan), or Chebyshev of
//               degree 8 over [hi/30, hi] when the last level is larger.
//
// The V-cycle is a fixed symmetric linear operator.  Each level is a CSR
// matrix kept on the device in FP64 and FP32; a row is summed by a group of
// w lanes (w the power of two that gives about four entries per lane, at
// most a warp), each lane over every w-th entry, then a fixed butterfly, so
// every result is deterministic.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "fsi_internal.cuh"

namespace fsi {

constexpr int kAmgMaxLevels = 16;
constexpr int64_t kAmgDirectMax = 600;
constexpr double kAmgThetaTet = 0.08, kAmgThetaHex = 0.02;
constexpr int kAmgNu = 2;
constexpr double kAmgLoRatio = 10.0;
constexpr int kAmgCoarseDegree = 8;
constexpr int kAmgPowerIts = 30;

struct AmgCsr {
    int64_t rows = 0, nnz = 0;
    int w = 1;  // lanes per row of the SpMV kernels: ~4 entries per lane
    int32_t *ptr = nullptr, *col = nullptr;
    double *v64 = nullptr;
    float *v32 = nullptr;
};

struct AmgLevel {
    int64_t n = 0;
    AmgCsr A, P, R;  // P: rows of this level -> next level; R = P^T
    double *dinv64 = nullptr;
    float *dinv32 = nullptr;
    double hi = 1.0;  // Chebyshev upper bound of D^-1 A
    // level vectors, 8 bytes per entry: right-hand side, solution, residual
    // (also a smoother x buffer), pre-smoothed iterate, two directions, x buffer
    void *b = nullptr, *x = nullptr, *r = nullptr, *t = nullptr, *d0 = nullptr,
         *d1 = nullptr, *xa = nullptr;
};

struct TetAmg {
    int nlev = 0;
    AmgLevel lev[kAmgMaxLevels];
    double kappa = 0.0;
    bool direct = false;
    int64_t nc = 0;
    double *inv64 = nullptr;
    float *inv32 = nullptr;
    bool built = false;
    std::vector<uint8_t> elim;      // elimination set of the built hierarchy
    std::vector<uint8_t> boundary;  // nodes on a boundary face
    int nv = 4;                     // corners per element: 4 tetrahedron, 8 hexahedron
    std::vector<double> Ae;         // per element nv x nv K + kappa M
    std::vector<int32_t> conn;      // [E][nv]
    std::vector<int64_t> nstart;    // node -> (element, corner) lists
    std::vector<int64_t> nslot;
};

namespace {

// ------------------------------------------------------------ host setup
struct HostCsr {
    int64_t rows = 0, cols = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
};

// K + kappa M of one linear tetrahedron: K_ab = V grad(l_a) . grad(l_b),
// M_ab = V (1 + delta_ab) / 20, V = |det J| / 6, J = [x1-x0, x2-x0, x3-x0];
// grad(l_{k+1}) is row k of J^-1 and grad(l_0) = -(the other three)
void element_matrix(const double x[4][3], double kappa, double *Ae)
{
    double J[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) J[i][k] = x[k + 1][i] - x[0][i];
    double C[3][3];  // cofactors
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    double g[4][3];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) g[k + 1][i] = C[i][k] / det;  // (J^-1)_{ki} = C_ik / det
    for (int i = 0; i < 3; ++i) g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
    const double V = std::fabs(det) / 6.0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            Ae[4 * a + b] = V * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]) +
                            kappa * V * (a == b ? 2.0 : 1.0) / 20.0;
}

// K + kappa M of one trilinear hexahedron, corner a at parent vertex
// (s_0, s_1, s_2) = (2(a&1)-1, 2((a>>1)&1)-1, 2((a>>2)&1)-1) of [-1, 1]^3,
// N_a = prod_k (1 + s_k xi_k) / 8: the integrals over the eight Gauss points
// xi_k = +-1/sqrt(3) (weights 1) with J_ik = dx_i/dxi_k,
// grad N_a = J^-T grad_xi N_a and dV = |det J| dxi
void hex_element_matrix(const double x[8][3], double kappa, double *Ae)
{
    const double g = 1.0 / std::sqrt(3.0);
    for (int q = 0; q < 64; ++q) Ae[q] = 0.0;
    for (int gp = 0; gp < 8; ++gp) {
        const double xi[3] = {(gp & 1) ? g : -g, (gp & 2) ? g : -g, (gp & 4) ? g : -g};
        double N[8], dN[8][3];
        for (int a = 0; a < 8; ++a) {
            double f[3], s[3];
            for (int k = 0; k < 3; ++k) {
                s[k] = ((a >> k) & 1) ? 1.0 : -1.0;
                f[k] = 0.5 * (1.0 + s[k] * xi[k]);
            }
            N[a] = f[0] * f[1] * f[2];
            dN[a][0] = 0.5 * s[0] * f[1] * f[2];
            dN[a][1] = 0.5 * s[1] * f[0] * f[2];
            dN[a][2] = 0.5 * s[2] * f[0] * f[1];
        }
        double J[3][3] = {};
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) J[i][k] += x[a][i] * dN[a][k];
        double C[3][3];  // cofactors: (J^-1)_{ki} = C_ik / det
        C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        double gx[8][3];  // (grad N_a)_i = sum_k (J^-1)_{ki} dN_a/dxi_k
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                gx[a][i] = (C[i][0] * dN[a][0] + C[i][1] * dN[a][1] + C[i][2] * dN[a][2]) / det;
        const double w = std::fabs(det);
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b)
                Ae[8 * a + b] += w * (gx[a][0] * gx[b][0] + gx[a][1] * gx[b][1] +
                                      gx[a][2] * gx[b][2] + kappa * N[a] * N[b]);
    }
}

// level-0 operator: rows assembled node by node from the node's element
// list (increasing element number), columns sorted; eliminated rows and
// columns keep only the diagonal
HostCsr assemble(const TetAmg &H, int64_t n)
{
    HostCsr A;
    A.rows = A.cols = n;
    A.ptr.assign((size_t)n + 1, 0);
    std::vector<int64_t> where((size_t)n, -1);
    std::vector<int32_t> cols;
    std::vector<double> vals;
    for (int64_t i = 0; i < n; ++i) {
        cols.clear();
        vals.clear();
        for (int64_t q = H.nstart[i]; q < H.nstart[i + 1]; ++q) {
            const int nv = H.nv;
            const int64_t e = H.nslot[q] / nv;
            const int a = (int)(H.nslot[q] % nv);
            for (int b = 0; b < nv; ++b) {
                const int32_t j = H.conn[nv * e + b];
                if (j != i && (H.elim[i] || H.elim[j])) continue;
                const double v = H.Ae[(int64_t)nv * nv * e + nv * a + b];
                if (where[j] < 0) {
                    where[j] = (int64_t)cols.size();
                    cols.push_back(j);
                    vals.push_back(v);
                } else {
                    vals[where[j]] += v;
                }
            }
        }
        if (where[i] < 0) {  // a node of no element: a unit row keeps A regular
            where[i] = (int64_t)cols.size();
            cols.push_back((int32_t)i);
            vals.push_back(1.0);
        }
        std::vector<int> order(cols.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        std::sort(order.begin(), order.end(), [&](int p, int q) { return cols[p] < cols[q]; });
        for (int k : order) {
            A.col.push_back(cols[k]);
            A.val.push_back(vals[k]);
        }
        for (int32_t j : cols) where[j] = -1;
        A.ptr[i + 1] = (int64_t)A.col.size();
    }
    return A;
}

std::vector<double> diagonal(const HostCsr &A)
{
    std::vector<double> d((size_t)A.rows, 0.0);
    for (int64_t i = 0; i < A.rows; ++i)
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
            if (A.col[q] == i) d[i] = A.val[q];
    return d;
}

// C = A B (Gustavson, rows in order, columns sorted)
HostCsr multiply(const HostCsr &A, const HostCsr &B)
{
    HostCsr C;
    C.rows = A.rows;
    C.cols = B.cols;
    C.ptr.assign((size_t)A.rows + 1, 0);
    std::vector<int64_t> where((size_t)B.cols, -1);
    std::vector<int32_t> cols;
    std::vector<double> vals;
    for (int64_t i = 0; i < A.rows; ++i) {
        cols.clear();
        vals.clear();
        for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
            const int32_t k = A.col[p];
            const double a = A.val[p];
            for (int64_t q = B.ptr[k]; q < B.ptr[k + 1]; ++q) {
                const int32_t j = B.col[q];
                if (where[j] < 0) {
                    where[j] = (int64_t)cols.size();
                    cols.push_back(j);
                    vals.push_back(a * B.val[q]);
                } else {
                    vals[where[j]] += a * B.val[q];
                }
            }
        }
        std::vector<int> order(cols.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        std::sort(order.begin(), order.end(), [&](int p, int q) { return cols[p] < cols[q]; });
        for (int k : order) {
            C.col.push_back(cols[k]);
            C.val.push_back(vals[k]);
        }
        for (int32_t j : cols) where[j] = -1;
        C.ptr[i + 1] = (int64_t)C.col.size();
    }
    return C;
}

HostCsr transpose(const HostCsr &A)
{
    HostCsr T;
    T.rows = A.cols;
    T.cols = A.rows;
    T.ptr.assign((size_t)T.rows + 1, 0);
    for (int32_t j : A.col) ++T.ptr[j + 1];
    for (int64_t r = 0; r < T.rows; ++r) T.ptr[r + 1] += T.ptr[r];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<int64_t> cur(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t i = 0; i < A.rows; ++i)
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
            const int64_t at = cur[A.col[q]]++;
            T.col[at] = (int32_t)i;
            T.val[at] = A.val[q];
        }
    return T;
}

// spectral radius of D^-1 A: power iteration on the symmetric D^-1/2 A D^-1/2
// from a fixed pseudo-random start (Rayleigh quotient of the last iterate),
// capped by the Gershgorin bound max_i sum_j |a_ij| / a_ii
double spectral_radius(const HostCsr &A, const std::vector<double> &d)
{
    const int64_t n = A.rows;
    double gersh = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += std::fabs(A.val[q]);
        gersh = std::max(gersh, s / d[i]);
    }
    std::vector<double> sd((size_t)n), v((size_t)n), w((size_t)n);
    for (int64_t i = 0; i < n; ++i) sd[i] = 1.0 / std::sqrt(d[i]);
    uint64_t state = 0x9E3779B97F4A7C15ull;
    for (int64_t i = 0; i < n; ++i) {
        state = state * 6364136223846793005ull + 1442695040888963407ull;
        v[i] = (double)(state >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    double lambda = 0.0;
    for (int it = 0; it < kAmgPowerIts; ++it) {
        double nv = 0.0;
        for (double x : v) nv += x * x;
        nv = std::sqrt(nv);
        if (!(nv > 0.0)) break;
        for (double &x : v) x /= nv;
        double vw = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += A.val[q] * sd[A.col[q]] * v[A.col[q]];
            w[i] = sd[i] * s;
            vw += v[i] * w[i];
        }
        lambda = vw;
        v.swap(w);
    }
    return std::min(std::max(lambda, 1e-300), gersh);
}

// aggregate number per node (-1: in none); returns the number of aggregates
int64_t aggregate(const HostCsr &A, const std::vector<double> &d, double theta,
                  std::vector<int32_t> &agg)
{
    const int64_t n = A.rows;
    std::vector<int64_t> sptr((size_t)n + 1, 0);
    std::vector<int32_t> scol;
    std::vector<double> sval;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
            const int32_t j = A.col[q];
            if (j == i) continue;
            if (std::fabs(A.val[q]) >= theta * std::sqrt(std::fabs(d[i] * d[j]))) {
                scol.push_back(j);
                sval.push_back(std::fabs(A.val[q]));
            }
        }
        sptr[i + 1] = (int64_t)scol.size();
    }
    const int32_t kFree = -1, kNone = -2;
    agg.assign((size_t)n, kFree);
    for (int64_t i = 0; i < n; ++i)
        if (sptr[i + 1] == sptr[i]) agg[i] = kNone;
    int32_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] != kFree) continue;
        bool all_free = true;
        for (int64_t q = sptr[i]; q < sptr[i + 1] && all_free; ++q) all_free = agg[scol[q]] == kFree;
        if (!all_free) continue;
        agg[i] = na;
        for (int64_t q = sptr[i]; q < sptr[i + 1]; ++q) agg[scol[q]] = na;
        ++na;
    }
    const std::vector<int32_t> first(agg);
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] != kFree) continue;
        double best = -1.0;
        for (int64_t q = sptr[i]; q < sptr[i + 1]; ++q)
            if (first[scol[q]] >= 0 && sval[q] > best) {
                best = sval[q];
                agg[i] = first[scol[q]];
            }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] != kFree) continue;
        agg[i] = na;
        for (int64_t q = sptr[i]; q < sptr[i + 1]; ++q)
            if (agg[scol[q]] == kFree) agg[scol[q]] = na;
        ++na;
    }
    for (int32_t &a : agg)
        if (a == kNone) a = -1;
    return na;
}

// P = (I - omega D^-1 A) P0
HostCsr smoothed_prolongator(const HostCsr &A, const std::vector<double> &d, double rho,
                             const std::vector<int32_t> &agg, int64_t na)
{
    HostCsr P0;
    P0.rows = A.rows;
    P0.cols = na;
    P0.ptr.assign((size_t)A.rows + 1, 0);
    for (int64_t i = 0; i < A.rows; ++i) {
        if (agg[i] >= 0) {
            P0.col.push_back(agg[i]);
            P0.val.push_back(1.0);
        }
        P0.ptr[i + 1] = (int64_t)P0.col.size();
    }
    HostCsr P = multiply(A, P0);  // A P0, rows hold every column of P0's row
    const double omega = 4.0 / (3.0 * rho);
    for (int64_t i = 0; i < A.rows; ++i)
        for (int64_t q = P.ptr[i]; q < P.ptr[i + 1]; ++q)
            P.val[q] = (P.col[q] == agg[i] ? 1.0 : 0.0) - omega * P.val[q] / d[i];
    return P;
}

// dense inverse of a small CSR matrix (Gauss-Jordan, partial pivoting, FP64)
bool dense_inverse(const HostCsr &A, std::vector<double> &inv)
{
    const int64_t n = A.rows, w = 2 * n;
    std::vector<double> a((size_t)n * w, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) a[i * w + A.col[q]] = A.val[q];
        a[i * w + n + i] = 1.0;
    }
    for (int64_t c = 0; c < n; ++c) {
        int64_t p = c;
        for (int64_t r = c + 1; r < n; ++r)
            if (std::fabs(a[r * w + c]) > std::fabs(a[p * w + c])) p = r;
        if (!(std::fabs(a[p * w + c]) > 0.0)) return false;
        if (p != c)
            for (int64_t q = 0; q < w; ++q) std::swap(a[p * w + q], a[c * w + q]);
        const double piv = 1.0 / a[c * w + c];
        for (int64_t q = 0; q < w; ++q) a[c * w + q] *= piv;
        for (int64_t r = 0; r < n; ++r)
            if (r != c) {
                const double f = a[r * w + c];
                if (f != 0.0)
                    for (int64_t q = 0; q < w; ++q) a[r * w + q] -= f * a[c * w + q];
            }
    }
    inv.assign((size_t)n * n, 0.0);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t c = 0; c < n; ++c) inv[r * n + c] = a[r * w + n + c];
    return true;
}

// ------------------------------------------------------------ device data
template <typename T> bool upload(T **dst, const T *src, size_t count)
{
    *dst = nullptr;
    if (count == 0) return true;
    if (cudaMalloc((void **)dst, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return false;
    }
    return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

bool upload_csr(AmgCsr &D, const HostCsr &H)
{
    D.rows = H.rows;
    D.nnz = (int64_t)H.col.size();
    D.w = 1;
    while (D.w < 32 && 4 * D.w * std::max<int64_t>(D.rows, 1) < D.nnz) D.w *= 2;
    std::vector<int32_t> ptr(H.ptr.begin(), H.ptr.end());
    std::vector<float> v32(H.val.begin(), H.val.end());
    int32_t dummy = 0;
    return upload(&D.ptr, ptr.data(), ptr.size()) &&
           upload(&D.col, H.col.empty() ? &dummy : H.col.data(), H.col.size()) &&
           upload(&D.v64, H.val.data(), H.val.size()) && upload(&D.v32, v32.data(), v32.size());
}

void free_csr(AmgCsr &D)
{
    cudaFree(D.ptr);
    cudaFree(D.col);
    cudaFree(D.v64);
    cudaFree(D.v32);
    D = AmgCsr{};
}

void free_levels(TetAmg &H)
{
    for (int l = 0; l < H.nlev; ++l) {
        AmgLevel &L = H.lev[l];
        free_csr(L.A);
        free_csr(L.P);
        free_csr(L.R);
        cudaFree(L.dinv64);
        cudaFree(L.dinv32);
        void *bufs[] = {L.b, L.x, L.r, L.t, L.d0, L.d1, L.xa};
        for (void *q : bufs) cudaFree(q);
        L = AmgLevel{};
    }
    cudaFree(H.inv64);
    cudaFree(H.inv32);
    H.inv64 = nullptr;
    H.inv32 = nullptr;
    H.nlev = 0;
    H.built = false;
}

// ------------------------------------------------------------ kernels
template <typename T> struct Csr {
    int64_t n;
    const int32_t *__restrict__ ptr;
    const int32_t *__restrict__ col;
    const T *__restrict__ val;
    int w;  // lanes per row
};

template <typename T> Csr<T> csr(const AmgCsr &A)
{
    return {A.rows, A.ptr, A.col,
            std::is_same<T, double>::value ? (const T *)A.v64 : (const T *)A.v32, A.w};
}
template <typename T> const T *dinv(const AmgLevel &L)
{
    return std::is_same<T, double>::value ? (const T *)L.dinv64 : (const T *)L.dinv32;
}

// Rows in groups of w lanes (w a power of two, <= 32): a warp takes 32 / w
// consecutive rows per pass, and every lane of a warp makes the same number
// of passes, so the shuffles of the row sums always see the whole warp.
struct RowGroups {
    int lane, sub;        // lane within the row's group, group within the warp
    int64_t base0, step;  // first row of the warp's first pass, rows per pass of the grid
};
__device__ __forceinline__ RowGroups row_groups(int w)
{
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int rpw = 32 / w;
    return {(int)(threadIdx.x & (w - 1)), (int)((threadIdx.x & 31) / w), warp * rpw,
            nwarps * rpw};
}

template <typename T>
__device__ __forceinline__ T val(const T *__restrict__ x, const T *__restrict__ d, int64_t q)
{
    return x ? (d ? x[q] + d[q] : x[q]) : d[q];
}

// (A v)_i, v = x + d (x == null: v = d; d == null: v = x): the row's lanes
// take every w-th entry, then a butterfly gives every lane the row sum (fixed
// order for a given w)
template <typename T>
__device__ __forceinline__ T row_apply(const Csr<T> &A, int64_t i, bool valid, int lane,
                                       const T *__restrict__ x, const T *__restrict__ d)
{
    T s = T(0);
    if (valid) {
        const int32_t q1 = A.ptr[i + 1];
        for (int32_t q = A.ptr[i] + lane; q < q1; q += A.w) s += A.val[q] * val(x, d, A.col[q]);
    }
    for (int o = A.w >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// y = b - A x (b == null: y = A x)
template <typename T>
__global__ void csr_apply_kernel(Csr<T> A, const T *__restrict__ x, const T *__restrict__ b,
                                 T *__restrict__ y)
{
    const RowGroups G = row_groups(A.w);
    const int lane = G.lane;
    for (int64_t base = G.base0; base < A.n; base += G.step) {
        const int64_t i = base + G.sub;
        const bool valid = i < A.n;
        const T ax = row_apply(A, i, valid, lane, x, (const T *)nullptr);
        if (valid && lane == 0) y[i] = b ? b[i] - ax : ax;
    }
}

// y += A x (prolongation: A = P, x coarse, y fine)
template <typename T>
__global__ void csr_apply_add_kernel(Csr<T> A, const T *__restrict__ x, T *__restrict__ y)
{
    const RowGroups G = row_groups(A.w);
    const int lane = G.lane;
    for (int64_t base = G.base0; base < A.n; base += G.step) {
        const int64_t i = base + G.sub;
        const bool valid = i < A.n;
        const T ax = row_apply(A, i, valid, lane, x, (const T *)nullptr);
        if (valid && lane == 0) y[i] += ax;
    }
}

// Chebyshev, first direction d0 = D^-1 (b - A x) / theta (x == null: x = 0);
// with x_out it writes x_out = x + d0 instead (degree 1)
template <typename T>
__global__ void amg_cheb0_kernel(Csr<T> A, const T *__restrict__ dinv, const T *__restrict__ b,
                                 const T *__restrict__ x, T inv_theta, T *__restrict__ d_out,
                                 T *__restrict__ x_out)
{
    const RowGroups G = row_groups(A.w);
    const int lane = G.lane;
    for (int64_t base = G.base0; base < A.n; base += G.step) {
        const int64_t i = base + G.sub;
        const bool valid = i < A.n;
        const T ax = x ? row_apply(A, i, valid, lane, x, (const T *)nullptr) : T(0);
        if (valid && lane == 0) {
            const T r = x ? b[i] - ax : b[i];
            const T d0 = inv_theta * r * dinv[i];
            if (x_out)
                x_out[i] = x ? x[i] + d0 : d0;
            else
                d_out[i] = d0;
        }
    }
}

// one Chebyshev step from (x, d): x' = x + d, d' = c1 d + c2 D^-1 (b - A x');
// writes (x', d'), or x' + d' into x_final on the last step
template <typename T>
__global__ void amg_cheb_step_kernel(Csr<T> A, const T *__restrict__ dinv, const T *__restrict__ b,
                                     const T *__restrict__ x, const T *__restrict__ d, T c1, T c2,
                                     T *__restrict__ x_next, T *__restrict__ d_next,
                                     T *__restrict__ x_final)
{
    const RowGroups G = row_groups(A.w);
    const int lane = G.lane;
    for (int64_t base = G.base0; base < A.n; base += G.step) {
        const int64_t i = base + G.sub;
        const bool valid = i < A.n;
        const T ax = row_apply(A, i, valid, lane, x, d);
        if (valid && lane == 0) {
            const T xk = val(x, d, i);
            const T r = b[i] - ax;
            const T dn = c1 * d[i] + c2 * (r * dinv[i]);
            if (x_final) {
                x_final[i] = xk + dn;
            } else {
                x_next[i] = xk;
                d_next[i] = dn;
            }
        }
    }
}

template <typename T> __global__ void amg_copy_kernel(int64_t n, const T *a, T *b)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// x = Ainv b on the coarsest level: one warp per row, fixed reduction order
template <typename T>
__global__ void amg_dense_kernel(int64_t nc, const T *__restrict__ Ainv, const T *__restrict__ b,
                                 T *__restrict__ x)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp; row < nc; row += nwarps) {
        T s = T(0);
        for (int64_t c = lane; c < nc; c += 32) s += Ainv[row * nc + c] * b[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[row] = s;
    }
}

int rows_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 16)); }
// blocks of 256 threads for n rows in groups of w lanes
int rows_grid(const AmgCsr &A) { return rows_grid(A.rows * A.w); }

template <typename T> T *vec(void *p) { return static_cast<T *>(p); }

template <typename T>
fsi_status chebyshev(fsi_mesh *m, int l, int degree, double lo, double hi, const T *b,
                     const T *x_in, T *x_out)
{
    AmgLevel &L = m->amg->lev[l];
    const Csr<T> A = csr<T>(L.A);
    const T *di = dinv<T>(L);
    cudaStream_t s = m->stream;
    const int g = rows_grid(L.A);
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), s1 = theta / delta;
    if (degree == 1) {
        amg_cheb0_kernel<T><<<g, 256, 0, s>>>(A, di, b, x_in, (T)(1.0 / theta), nullptr, x_out);
        return check_launch("pressure AMG smoother");
    }
    T *dbuf[2] = {vec<T>(L.d0), vec<T>(L.d1)}, *xbuf[2] = {vec<T>(L.xa), vec<T>(L.r)};
    amg_cheb0_kernel<T><<<g, 256, 0, s>>>(A, di, b, x_in, (T)(1.0 / theta), dbuf[0], nullptr);
    const T *xc = x_in;
    const T *dc = dbuf[0];
    double rho = 1.0 / s1;
    for (int it = 1; it < degree; ++it) {
        const double rho_new = 1.0 / (2.0 * s1 - rho);
        const T c1 = (T)(rho_new * rho), c2 = (T)(2.0 * rho_new / delta);
        const bool last = it == degree - 1;
        T *xn = xbuf[it & 1], *dn = dbuf[it & 1];
        amg_cheb_step_kernel<T><<<g, 256, 0, s>>>(A, di, b, xc, dc, c1, c2, last ? nullptr : xn,
                                                  last ? nullptr : dn, last ? x_out : nullptr);
        xc = xn;
        dc = dn;
        rho = rho_new;
    }
    return check_launch("pressure AMG smoother");
}

template <typename T> fsi_status coarse_solve(fsi_mesh *m, const T *b, T *x)
{
    TetAmg &H = *m->amg;
    const int l = H.nlev - 1;
    if (H.direct) {
        const T *inv = std::is_same<T, double>::value ? (const T *)H.inv64 : (const T *)H.inv32;
        const int blocks = (int)std::min<int64_t>((H.nc + 7) / 8, sm_count() * 8);
        amg_dense_kernel<T><<<blocks, 256, 0, m->stream>>>(H.nc, inv, b, x);
        return check_launch("pressure AMG coarse solve");
    }
    return chebyshev<T>(m, l, kAmgCoarseDegree, H.lev[l].hi / 30.0, H.lev[l].hi, b, nullptr, x);
}

template <typename T> fsi_status vcycle_level(fsi_mesh *m, int l, const T *b, T *x)
{
    TetAmg &H = *m->amg;
    if (l == H.nlev - 1) return coarse_solve<T>(m, b, x);
    AmgLevel &L = H.lev[l], &Lc = H.lev[l + 1];
    const double hi = L.hi, lo = hi / kAmgLoRatio;
    T *t = vec<T>(L.t);
    FSI_TRY(chebyshev<T>(m, l, kAmgNu, lo, hi, b, (const T *)nullptr, t));
    csr_apply_kernel<T><<<rows_grid(L.A), 256, 0, m->stream>>>(csr<T>(L.A), t, b, vec<T>(L.r));
    csr_apply_kernel<T><<<rows_grid(L.R), 256, 0, m->stream>>>(csr<T>(L.R), vec<T>(L.r),
                                                                 (const T *)nullptr, vec<T>(Lc.b));
    FSI_TRY(check_launch("pressure AMG restrict"));
    FSI_TRY(vcycle_level<T>(m, l + 1, vec<T>(Lc.b), vec<T>(Lc.x)));
    csr_apply_add_kernel<T><<<rows_grid(L.P), 256, 0, m->stream>>>(csr<T>(L.P), vec<T>(Lc.x), t);
    FSI_TRY(check_launch("pressure AMG prolong"));
    return chebyshev<T>(m, l, kAmgNu, lo, hi, b, t, x);
}

// node -> (element, corner) lists of the connectivity, elements in
// increasing order
void node_lists(TetAmg &H, int64_t n)
{
    H.nstart.assign((size_t)n + 1, 0);
    for (int32_t v : H.conn) ++H.nstart[v + 1];
    for (int64_t i = 0; i < n; ++i) H.nstart[i + 1] += H.nstart[i];
    H.nslot.resize(H.conn.size());
    std::vector<int64_t> cur(H.nstart.begin(), H.nstart.end() - 1);
    for (int64_t s = 0; s < (int64_t)H.conn.size(); ++s) H.nslot[cur[H.conn[s]]++] = s;
}

double shift_for(const double lo[3], const double hi[3])
{
    double Lmax = 0.0;
    for (int d = 0; d < 3; ++d) Lmax = std::max(Lmax, hi[d] - lo[d]);
    const double q = 3.14159265358979323846 / (2.0 * Lmax);
    return q * q;
}

// host data of the structured grid: node (i, j, k) is i + (Nx+1)(j + (Ny+1)k),
// element (i, j, k) is i + Nx(j + Ny k) with corner a at node
// (i + (a&1), j + ((a>>1)&1), k + ((a>>2)&1)); coordinates from the mapped
// table when set, else x0 + i h; boundary nodes lie on the box's faces
fsi_status load_grid(fsi_mesh *m, TetAmg &H)
{
    const int32_t *N = m->grid.N;
    const int64_t NX1 = N[0] + 1, NY1 = N[1] + 1, NZ1 = N[2] + 1;
    const int64_t n = m->n_nodes, E = m->n_elems;
    std::vector<double> X((size_t)n * 3);
    if (m->coords64) {
        std::vector<double> C4((size_t)n * 4);
        FSI_CUDA(cudaMemcpyAsync(C4.data(), m->coords64, C4.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, m->stream),
                 "memcpy");
        FSI_CUDA(cudaStreamSynchronize(m->stream), "sync");
        for (int64_t v = 0; v < n; ++v)
            for (int d = 0; d < 3; ++d) X[3 * v + d] = C4[4 * v + d];
    } else {
        for (int64_t k = 0; k < NZ1; ++k)
            for (int64_t j = 0; j < NY1; ++j)
                for (int64_t i = 0; i < NX1; ++i) {
                    const int64_t v = i + NX1 * (j + NY1 * k);
                    X[3 * v] = m->grid.x0[0] + (double)i * m->grid.h[0];
                    X[3 * v + 1] = m->grid.x0[1] + (double)j * m->grid.h[1];
                    X[3 * v + 2] = m->grid.x0[2] + (double)k * m->grid.h[2];
                }
    }
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = X[d];
    for (int64_t v = 0; v < n; ++v)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], X[3 * v + d]);
            hi[d] = std::max(hi[d], X[3 * v + d]);
        }
    H.kappa = shift_for(lo, hi);
    H.nv = 8;
    H.conn.resize((size_t)E * 8);
    H.Ae.resize((size_t)E * 64);
    for (int64_t k = 0; k < N[2]; ++k)
        for (int64_t j = 0; j < N[1]; ++j)
            for (int64_t i = 0; i < N[0]; ++i) {
                const int64_t e = i + N[0] * (j + N[1] * k);
                double x[8][3];
                for (int a = 0; a < 8; ++a) {
                    const int64_t v = (i + (a & 1)) + NX1 * ((j + ((a >> 1) & 1)) +
                                                             NY1 * (k + ((a >> 2) & 1)));
                    H.conn[8 * e + a] = (int32_t)v;
                    for (int d = 0; d < 3; ++d) x[a][d] = X[3 * v + d];
                }
                hex_element_matrix(x, H.kappa, &H.Ae[64 * e]);
            }
    node_lists(H, n);
    H.boundary.assign((size_t)n, 0);
    for (int64_t k = 0; k < NZ1; ++k)
        for (int64_t j = 0; j < NY1; ++j)
            for (int64_t i = 0; i < NX1; ++i)
                H.boundary[i + NX1 * (j + NY1 * k)] = i == 0 || i == N[0] || j == 0 ||
                                                      j == N[1] || k == 0 || k == N[2];
    return FSI_OK;
}

// host data of the tetrahedral mesh: element matrices, node lists, boundary nodes
fsi_status load_mesh(fsi_mesh *m, TetAmg &H)
{
    std::vector<double> X;
    double lo[3], hi[3];
    FSI_TRY(tet_download(m->tet, X, H.conn, lo, hi));
    const int64_t n = m->n_nodes, E = (int64_t)H.conn.size() / 4;
    H.kappa = shift_for(lo, hi);
    H.nv = 4;
    H.Ae.resize((size_t)E * 16);
    for (int64_t e = 0; e < E; ++e) {
        double x[4][3];
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) x[a][i] = X[3 * (int64_t)H.conn[4 * e + a] + i];
        element_matrix(x, H.kappa, &H.Ae[16 * e]);
    }
    node_lists(H, n);
    // boundary faces: the faces (sorted node triples) that one element holds
    struct Face {
        int32_t v[3];
        bool operator<(const Face &o) const
        {
            return v[0] != o.v[0] ? v[0] < o.v[0] : (v[1] != o.v[1] ? v[1] < o.v[1] : v[2] < o.v[2]);
        }
        bool operator==(const Face &o) const
        {
            return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2];
        }
    };
    std::vector<Face> faces((size_t)E * 4);
    for (int64_t e = 0; e < E; ++e)
        for (int f = 0; f < 4; ++f) {
            Face F;
            int k = 0;
            for (int a = 0; a < 4; ++a)
                if (a != f) F.v[k++] = H.conn[4 * e + a];
            std::sort(F.v, F.v + 3);
            faces[4 * e + f] = F;
        }
    std::sort(faces.begin(), faces.end());
    H.boundary.assign((size_t)n, 0);
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j] == faces[i]) ++j;
        if (j - i == 1)
            for (int k = 0; k < 3; ++k) H.boundary[faces[i].v[k]] = 1;
        i = j;
    }
    return FSI_OK;
}

fsi_status ensure_host(fsi_mesh *m)
{
    FSI_TRY(validate_mesh(m));
    if (!uses_amg(m))
        return set_error(FSI_ERR_ARG, "pressure AMG: not selected for this structured grid "
                                      "(fsi_pressure_use_amg)");
    if (m->amg) return FSI_OK;
    TetAmg *H = new (std::nothrow) TetAmg();
    if (!H) return set_error(FSI_ERR_OOM, "host allocation of the pressure AMG failed");
    m->amg = H;
    fsi_status st = m->tet ? load_mesh(m, *H) : load_grid(m, *H);
    if (st != FSI_OK) {
        delete H;
        m->amg = nullptr;
        return st;
    }
    H->elim.assign((size_t)m->n_nodes, 0);
    return FSI_OK;
}

// the hierarchy for H.elim
fsi_status build(fsi_mesh *m)
{
    TetAmg &H = *m->amg;
    // device buffers of the old hierarchy may be in use by queued work
    FSI_CUDA(cudaStreamSynchronize(m->stream), "sync");
    free_levels(H);
    std::vector<HostCsr> A(1), P;
    A[0] = assemble(H, m->n_nodes);
    std::vector<std::vector<double>> D(1, diagonal(A[0]));
    std::vector<double> rho(1, spectral_radius(A[0], D[0]));
    while ((int)A.size() < kAmgMaxLevels && A.back().rows > kAmgDirectMax) {
        const HostCsr &Af = A.back();
        std::vector<int32_t> agg;
        const int64_t na = aggregate(Af, D.back(), H.nv == 8 ? kAmgThetaHex : kAmgThetaTet, agg);
        if (na == 0 || (double)na * 1.25 > (double)Af.rows) break;
        HostCsr Pl = smoothed_prolongator(Af, D.back(), rho.back(), agg, na);
        HostCsr Rl = transpose(Pl);
        HostCsr Ac = multiply(Rl, multiply(Af, Pl));
        P.push_back(std::move(Pl));
        A.push_back(std::move(Ac));
        D.push_back(diagonal(A.back()));
        rho.push_back(spectral_radius(A.back(), D.back()));
    }
    for (const HostCsr &M : A)
        if ((int64_t)M.col.size() >= INT32_MAX)
            return set_error(FSI_ERR_ARG, "pressure AMG: a level has 2^31 or more entries");
    H.nlev = (int)A.size();
    bool ok = true;
    for (int l = 0; l < H.nlev && ok; ++l) {
        AmgLevel &L = H.lev[l];
        L.n = A[l].rows;
        L.hi = 1.1 * rho[l];
        std::vector<double> di64((size_t)L.n);
        for (int64_t i = 0; i < L.n; ++i) di64[i] = 1.0 / D[l][i];
        std::vector<float> di32(di64.begin(), di64.end());
        ok = upload_csr(L.A, A[l]) && upload(&L.dinv64, di64.data(), di64.size()) &&
             upload(&L.dinv32, di32.data(), di32.size());
        if (ok && l + 1 < H.nlev) ok = upload_csr(L.P, P[l]) && upload_csr(L.R, transpose(P[l]));
        void **bufs[] = {&L.b, &L.x, &L.r, &L.t, &L.d0, &L.d1, &L.xa};
        for (void **b : bufs) {
            if (!ok) break;
            if (cudaMalloc(b, (size_t)std::max<int64_t>(L.n, 1) * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                *b = nullptr;
                ok = false;
            }
        }
    }
    if (!ok) {
        free_levels(H);
        return set_error(FSI_ERR_OOM, "pressure AMG: device allocation or copy failed");
    }
    const HostCsr &C = A.back();
    H.nc = C.rows;
    H.direct = C.rows <= kAmgDirectMax;
    if (H.direct) {
        std::vector<double> inv;
        if (!dense_inverse(C, inv)) {
            free_levels(H);
            return set_error(FSI_ERR_ARG, "pressure AMG: singular coarse operator");
        }
        std::vector<float> inv32(inv.begin(), inv.end());
        if (!upload(&H.inv64, inv.data(), inv.size()) ||
            !upload(&H.inv32, inv32.data(), inv32.size())) {
            free_levels(H);
            return set_error(FSI_ERR_OOM, "pressure AMG: device allocation or copy failed");
        }
    }
    H.built = true;
    return FSI_OK;
}

fsi_status ensure_built(fsi_mesh *m)
{
    FSI_TRY(ensure_host(m));
    return m->amg->built ? FSI_OK : build(m);
}

fsi_status check_prec(fsi_prec p)
{
    if (p != FSI_F64 && p != FSI_F32)
        return set_error(FSI_ERR_ARG, "pressure operator: precision must be FSI_F64 or FSI_F32");
    return FSI_OK;
}

fsi_status check_level(fsi_mesh *m, int level, bool need_coarser)
{
    if (level < 0 || level >= m->amg->nlev || (need_coarser && level + 1 >= m->amg->nlev))
        return set_error(FSI_ERR_ARG, "pressure operator: level %d out of range", level);
    return FSI_OK;
}

}  // namespace

void destroy_amg(fsi_mesh *m)
{
    if (!m->amg) return;
    free_levels(*m->amg);
    delete m->amg;
    m->amg = nullptr;
}

fsi_status amg_set_eliminated(fsi_mesh *m, const std::vector<uint8_t> &elim)
{
    FSI_TRY(ensure_host(m));
    TetAmg &H = *m->amg;
    if (H.built && elim == H.elim) return FSI_OK;
    H.elim = elim;
    return build(m);
}

fsi_status amg_set_from_mask(fsi_mesh *m, const uint8_t *mask)
{
    FSI_TRY(ensure_host(m));
    const int64_t n = m->n_nodes;
    std::vector<uint8_t> hm;
    if (mask) {
        hm.resize((size_t)n * 4);
        FSI_CUDA(cudaMemcpyAsync(hm.data(), mask, hm.size(), cudaMemcpyDeviceToHost, m->stream),
                 "memcpy");
        FSI_CUDA(cudaStreamSynchronize(m->stream), "sync");
    }
    std::vector<uint8_t> elim((size_t)n, 0);
    const std::vector<uint8_t> &bd = m->amg->boundary;
    for (int64_t i = 0; i < n; ++i) {
        const bool vfree = !mask || !(hm[4 * i] | hm[4 * i + 1] | hm[4 * i + 2]);
        const bool pfixed = mask && hm[4 * i + 3];
        elim[i] = (bd[i] && vfree) || pfixed;
    }
    return amg_set_eliminated(m, elim);
}

template <typename T> fsi_status amg_vcycle(fsi_mesh *m, const T *b, T *x)
{
    FSI_TRY(ensure_built(m));
    return vcycle_level<T>(m, 0, b, x);
}
template fsi_status amg_vcycle<double>(fsi_mesh *, const double *, double *);
template fsi_status amg_vcycle<float>(fsi_mesh *, const float *, float *);

void *amg_fine_buffer(fsi_mesh *m, int which)
{
    return which == 0 ? m->amg->lev[0].b : m->amg->lev[0].x;
}

fsi_status amg_level_sizes(fsi_mesh *m, int32_t *n_levels, int64_t *n)
{
    FSI_TRY(ensure_built(m));
    *n_levels = m->amg->nlev;
    if (n)
        for (int l = 0; l < m->amg->nlev; ++l) n[l] = m->amg->lev[l].n;
    return FSI_OK;
}

fsi_status amg_apply(fsi_mesh *m, fsi_prec prec, int level, const void *x, void *y)
{
    FSI_TRY(check_prec(prec));
    FSI_TRY(ensure_built(m));
    FSI_TRY(check_level(m, level, false));
    const AmgLevel &L = m->amg->lev[level];
    if (prec == FSI_F64)
        csr_apply_kernel<double><<<rows_grid(L.A), 256, 0, m->stream>>>(
            csr<double>(L.A), (const double *)x, nullptr, (double *)y);
    else
        csr_apply_kernel<float><<<rows_grid(L.A), 256, 0, m->stream>>>(
            csr<float>(L.A), (const float *)x, nullptr, (float *)y);
    return check_launch("pressure AMG apply");
}

fsi_status amg_restrict(fsi_mesh *m, fsi_prec prec, int level, const void *r, void *b)
{
    FSI_TRY(check_prec(prec));
    FSI_TRY(ensure_built(m));
    FSI_TRY(check_level(m, level, true));
    const AmgLevel &L = m->amg->lev[level];
    const int g = rows_grid(L.R);
    if (prec == FSI_F64)
        csr_apply_kernel<double><<<g, 256, 0, m->stream>>>(csr<double>(L.R), (const double *)r,
                                                           nullptr, (double *)b);
    else
        csr_apply_kernel<float><<<g, 256, 0, m->stream>>>(csr<float>(L.R), (const float *)r,
                                                          nullptr, (float *)b);
    return check_launch("pressure AMG restrict");
}

fsi_status amg_prolong_add(fsi_mesh *m, fsi_prec prec, int level, const void *xc, void *x)
{
    FSI_TRY(check_prec(prec));
    FSI_TRY(ensure_built(m));
    FSI_TRY(check_level(m, level, true));
    const AmgLevel &L = m->amg->lev[level];
    if (prec == FSI_F64)
        csr_apply_add_kernel<double><<<rows_grid(L.P), 256, 0, m->stream>>>(
            csr<double>(L.P), (const double *)xc, (double *)x);
    else
        csr_apply_add_kernel<float><<<rows_grid(L.P), 256, 0, m->stream>>>(
            csr<float>(L.P), (const float *)xc, (float *)x);
    return check_launch("pressure AMG prolong");
}

fsi_status amg_smooth(fsi_mesh *m, fsi_prec prec, int level, int degree, const void *b, void *x,
                      int from_zero)
{
    FSI_TRY(check_prec(prec));
    FSI_TRY(ensure_built(m));
    FSI_TRY(check_level(m, level, false));
    AmgLevel &L = m->amg->lev[level];
    const double hi = L.hi, lo = hi / kAmgLoRatio;
    if (prec == FSI_F64) {
        const double *xin = nullptr;
        if (!from_zero) {
            amg_copy_kernel<double><<<rows_grid(L.n), 256, 0, m->stream>>>(L.n, (const double *)x,
                                                                          vec<double>(L.t));
            xin = vec<double>(L.t);
        }
        return chebyshev<double>(m, level, degree, lo, hi, (const double *)b, xin, (double *)x);
    }
    const float *xin = nullptr;
    if (!from_zero) {
        amg_copy_kernel<float><<<rows_grid(L.n), 256, 0, m->stream>>>(L.n, (const float *)x,
                                                                     vec<float>(L.t));
        xin = vec<float>(L.t);
    }
    return chebyshev<float>(m, level, degree, lo, hi, (const float *)b, xin, (float *)x);
}

}  // namespace fsi
