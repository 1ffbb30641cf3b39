// pmg.cu -- pressure block of the Schur-complement block preconditioner
// (Sec. 2.4 solves the reduced system with block preconditioners built from
// its sub-matrices).  For the saddle-point blocks [[A, B], [C, D]] of the
// linearised fluid system with a mass-dominated velocity block
// A ~ alpha_m rho M, the pressure Schur complement D - C A^{-1} B acts like
// sigma K, K the Q1 stiffness matrix of the pressure space and
// sigma = alpha_f gamma dt / (alpha_m rho).  The preconditioner replaces it by
// sigma (K + kappa M), kappa = (pi / (2 L))^2 with L the largest extent of the
// grid (M the Q1 mass matrix; the shift keeps the operator non-singular where
// only Neumann conditions bound the pressure).  On faces of the box where the
// velocity is free (traction-free outflow) the true Schur complement acts like
// a Dirichlet problem for the pressure, so the nodes of such faces are
// eliminated (rows and columns dropped, diagonal kept; the restricted
// right-hand side is zeroed there).  The approximation is inverted with one
// geometric multigrid V-cycle on the uniform grid:
//
//   levels     the mesh grid, then every other node while all N_d are even and
//              the grid has more than 125 nodes;
//   operator   K + kappa M applied matrix-free: on a uniform grid both are
//              tensor products of the 1D linear-element matrices
//              M1 = h/6 [1 4 1] (h/3 on boundary nodes) and
//              K1 = 1/h [-1 2 -1] (1/h on boundary nodes):
//              K = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1;
//   transfer   trilinear interpolation P, restriction P^T (weights 1, 1/2);
//              the coarse operators equal P^T A P (Galerkin) exactly;
//   smoother   Chebyshev semi-iteration of degree 2 on D^{-1} A over
//              [hi/4, hi], hi = 1.1 x the largest symbol/diagonal ratio over
//              the modes theta_d in {0, pi} (pre- and post-smoothing);
//   coarsest   a dense inverse (<= 1000 nodes, built once on the host in
//              FP64) or, on grids that do not coarsen, Chebyshev degree 8 over
//              [hi/30, hi].
//
// The V-cycle is a fixed linear operator (symmetric), so it can precondition
// plain GMRES.  Every kernel is one thread per node, deterministic; FP64 or
// FP32 arithmetic follows the caller's precision.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "fsi_internal.cuh"

namespace fsi {

constexpr int kPmgMaxLevels = 16;
constexpr int kPmgNu = 2;
constexpr int kPmgCoarseDegree = 8;
constexpr int64_t kPmgDirectMax = 1000;
constexpr int64_t kPmgMinCoarsen = 125;

struct PmgLevel {
    int N[3];
    double h[3];
    int64_t n;
    double hi;          // Chebyshev upper bound of D^{-1} A
    // level vectors, 8 bytes per entry (either precision fits): right-hand
    // side, solution, residual (also the second x buffer of the smoother),
    // pre-smoothed iterate, two smoother directions, one more x buffer
    void *b, *x, *r, *t, *d0, *d1, *xa;
};

struct PressureMG {
    int nlev = 0;
    PmgLevel lev[kPmgMaxLevels];
    double kappa = 0.0;
    int faces[6] = {0, 0, 0, 0, 0, 0};  // eliminated faces x0, x1, y0, y1, z0, z1
    bool direct = false;
    int64_t nc = 0;
    double *inv64 = nullptr;  // [nc][nc]
    float *inv32 = nullptr;
};

namespace {

// 1D coefficients of a level in the working type: mass and stiffness
// entries of interior / boundary diagonals and of the off-diagonals.
template <typename T> struct Axis {
    int N;
    T m_in, m_bd, m_off, k_in, k_bd, k_off;
};

template <typename T> struct LevelArgs {
    Axis<T> a[3];
    T kappa;
    int NX1, NY1, NZ1;
    int faces[6];
};

template <typename T> LevelArgs<T> level_args(const PressureMG &P, int l)
{
    const PmgLevel &L = P.lev[l];
    LevelArgs<T> A;
    for (int d = 0; d < 3; ++d) {
        const double h = L.h[d];
        A.a[d] = {L.N[d], (T)(2.0 * h / 3.0), (T)(h / 3.0), (T)(h / 6.0),
                  (T)(2.0 / h), (T)(1.0 / h), (T)(-1.0 / h)};
    }
    A.kappa = (T)P.kappa;
    A.NX1 = L.N[0] + 1;
    A.NY1 = L.N[1] + 1;
    A.NZ1 = L.N[2] + 1;
    for (int f = 0; f < 6; ++f) A.faces[f] = P.faces[f];
    return A;
}

// node (i, j, k) lies on an eliminated face
template <typename T>
__device__ __forceinline__ bool eliminated(const LevelArgs<T> &L, int i, int j, int k)
{
    return (L.faces[0] && i == 0) || (L.faces[1] && i == L.NX1 - 1) ||
           (L.faces[2] && j == 0) || (L.faces[3] && j == L.NY1 - 1) ||
           (L.faces[4] && k == 0) || (L.faces[5] && k == L.NZ1 - 1);
}

// entries (mass, stiffness) of row i, column i + d (|d| <= 1, in range)
template <typename T>
__device__ __forceinline__ void coef(const Axis<T> &a, int i, int d, T &m, T &k)
{
    if (d == 0) {
        const bool bd = (i == 0) || (i == a.N);
        m = bd ? a.m_bd : a.m_in;
        k = bd ? a.k_bd : a.k_in;
    } else {
        m = a.m_off;
        k = a.k_off;
    }
}

template <typename T> __device__ __forceinline__ T diag_of(const LevelArgs<T> &L, int i, int j, int k)
{
    T mx, kx, my, ky, mz, kz;
    coef(L.a[0], i, 0, mx, kx);
    coef(L.a[1], j, 0, my, ky);
    coef(L.a[2], k, 0, mz, kz);
    return kx * my * mz + mx * ky * mz + mx * my * kz + L.kappa * mx * my * mz;
}

// v = x + d at a node (x == null: v = d; d == null: v = x)
template <typename T>
__device__ __forceinline__ T val(const T *__restrict__ x, const T *__restrict__ d, int64_t q)
{
    return x ? (d ? x[q] + d[q] : x[q]) : d[q];
}

// One thread per (i, j) column on a 3D launch, x and y from the block and
// thread indices, striding over the planes k from the grid's z index (no
// per-node division; a CTA does several planes, so tiny CTAs do not make the
// CTA launches the limit).
#define NODE3(L, i, j, k)                                                                   \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;                                 \
    const int j = blockIdx.y * blockDim.y + threadIdx.y;                                 \
    if (i >= (L).NX1 || j >= (L).NY1) return;                                            \
    for (int k = blockIdx.z; k < (L).NZ1; k += gridDim.z)

// Chebyshev, first direction from x = 0: d0 = D^{-1} b / theta, or with
// x_out (degree 1) x_out = d0.  (From a nonzero x the first direction needs
// A x: march_kernel in kMarchCheb0 mode.)
template <typename T>
__global__ void cheb0_kernel(LevelArgs<T> L, const T *__restrict__ b, T inv_theta,
                             T *__restrict__ d_out, T *__restrict__ x_out)
{
    NODE3(L, i, j, k)
    {
        const int64_t node = i + (int64_t)L.NX1 * (j + (int64_t)L.NY1 * k);
        const T d0 = inv_theta * b[node] / diag_of(L, i, j, k);
        if (x_out)
            x_out[node] = d0;
        else
            d_out[node] = d0;
    }
}

// ---------------------------------------------------------------- z-marching stencil
// The operator A = K + kappa M of a level is a tensor product of 1D Q1 rows
// (stiffness k, mass m per axis), so (A v)_node = sum_dk [P(k+dk) mz(dk) +
// Q(k+dk) kz(dk)] with, per plane k', P = Ax + By + kappa C and Q = C, where
// Ax = sum_dj sK_x(j+dj) my(dj), By = sum_dj sM_x(j+dj) ky(dj), C = sum_dj
// sM_x(j+dj) my(dj), and sK_x / sM_x the 1D stiffness / mass rows along x.
// A CTA of 32 x 8 threads owns a 32 x 8 column of nodes and marches up kz
// planes (as many as leave about 16 CTAs per SM, 2 to 16): per plane it
// stages v (with a one-node
// halo, zero outside the grid and on eliminated nodes, whose columns A does
// not have) in shared memory, forms the x rows once per position, and each
// thread folds its 3 x 3 neighbourhood into (P, Q) for the plane; the z fold
// uses the three most recent planes held in registers.  The next plane's
// loads are issued before the current plane is folded, so their latency
// overlaps the work.  Every v is read once per plane (plus halos) instead of
// 27 times, and the per-node work is ~30 operations.  Rows of eliminated
// nodes keep only the diagonal.  The sums run in a fixed order
// (deterministic).  (One thread per column marching without shared memory,
// reading its 3 x 3 neighbourhood through L1, measured 1.8x slower; two
// rows per thread, 8 apart, measured 1.3x slower at 129^3: 88-94 registers
// leave 2 CTAs per SM.)  The source of v (x, d or x + d) is a template
// parameter, so no pass tests for null vectors per load.
constexpr int kMarchX = 32, kMarchTY = 8, kMarchRows = 1;    // threads x, threads y, rows per thread
constexpr int kMarchY = kMarchTY * kMarchRows;                   // node rows per CTA
constexpr int kMarchThreads = kMarchX * kMarchTY;
constexpr int kStage = (kMarchY + 2) * (kMarchX + 2);            // staged values per plane
constexpr int kStagePer = (kStage + kMarchThreads - 1) / kMarchThreads;
constexpr int kXRows = (kMarchY + 2) * kMarchX;                  // x-row positions per plane
constexpr int kXRowPer = (kXRows + kMarchThreads - 1) / kMarchThreads;

template <typename T> struct March {
    const T *x, *d;  // v = x + d (VX selects which are present)
    const T *b;
    T c1, c2, inv_theta;
    T *y, *x_next, *d_next, *x_final;
    int kz;          // planes per CTA
    // with z4 (a step's x_final): the result goes to z4[4 node + 3] as
    // x_final * inv_sigma, or v4[4 node + 3] where m4[4 node + 3] is set
    T *z4;
    const T *v4;
    const uint8_t *m4;
    T inv_sigma;
};

enum MarchMode { kMarchApply = 0, kMarchCheb0 = 1, kMarchStep = 2 };
// the vector v the stencil acts on: d alone, x alone, x + d, or (kVb) the
// first Chebyshev direction from x = 0, d0 = b / (theta D), formed from b at
// every staged node (so no pass writes d0 first)
enum MarchSource { kVd = 0, kVx = 1, kVxd = 2, kVb = 3 };

template <typename T>
__device__ __forceinline__ T md_of(const Axis<T> &a, int i)
{
    return (i == 0 || i == a.N) ? a.m_bd : a.m_in;
}
template <typename T>
__device__ __forceinline__ T kd_of(const Axis<T> &a, int i)
{
    return (i == 0 || i == a.N) ? a.k_bd : a.k_in;
}
template <typename T, int VX> __device__ __forceinline__ T vsrc(const March<T> &M, int64_t q)
{
    if constexpr (VX == kVd) return M.d[q];
    else if constexpr (VX == kVx) return M.x[q];
    else return M.x[q] + M.d[q];
}

template <typename T, int MODE, int VX>
__global__ void __launch_bounds__(kMarchThreads) march_kernel(LevelArgs<T> L, March<T> M)
{
    __shared__ T vt[kStage];                      // [kMarchY + 2][kMarchX + 2]
    __shared__ T sk[kXRows], sm[kXRows];          // [kMarchY + 2][kMarchX]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kMarchX * ty;
    const int i0 = blockIdx.x * kMarchX, j0 = blockIdx.y * kMarchY, k0 = blockIdx.z * M.kz;
    const int i = i0 + tx;
    const Axis<T> &ax = L.a[0], &ay = L.a[1], &az = L.a[2];
    const int64_t plane_n = (int64_t)L.NX1 * L.NY1;
    // per thread, once: the staged slots' in-plane offsets and masks (x, y
    // faces), the x-row slots' centre coefficients and staged indices
    int64_t s_off[kStagePer];
    bool s_in[kStagePer];
    // kVb: 1/D of the staged column's nodes on an interior / boundary plane
    T s_iDi[kStagePer], s_iDb[kStagePer];
#pragma unroll
    for (int r = 0; r < kStagePer; ++r) {
        const int q = tid + r * kMarchThreads;
        const int gi = i0 - 1 + q % (kMarchX + 2), gj = j0 - 1 + q / (kMarchX + 2);
        s_in[r] = q < kStage && gi >= 0 && gj >= 0 && gi < L.NX1 && gj < L.NY1 &&
                  !((L.faces[0] && gi == 0) || (L.faces[1] && gi == L.NX1 - 1) ||
                    (L.faces[2] && gj == 0) || (L.faces[3] && gj == L.NY1 - 1));
        s_off[r] = gi + (int64_t)L.NX1 * gj;
        if constexpr (VX == kVb) {
            const T mx = md_of(L.a[0], gi), kx = kd_of(L.a[0], gi);
            const T my = md_of(L.a[1], gj), ky = kd_of(L.a[1], gj);
            const T a1 = kx * my + mx * ky + L.kappa * mx * my, a2 = mx * my;
            s_iDi[r] = T(1) / (a1 * L.a[2].m_in + a2 * L.a[2].k_in);
            s_iDb[r] = T(1) / (a1 * L.a[2].m_bd + a2 * L.a[2].k_bd);
        }
    }
    T x_k[kXRowPer], x_m[kXRowPer];
    int x_v[kXRowPer];
#pragma unroll
    for (int r = 0; r < kXRowPer; ++r) {
        const int q = tid + r * kMarchThreads;
        const int cx = q % kMarchX, cy = q / kMarchX;
        x_k[r] = kd_of(ax, i0 + cx);
        x_m[r] = md_of(ax, i0 + cx);
        x_v[r] = cy * (kMarchX + 2) + cx;
    }
    // this thread's nodes (i, j0 + ty + kMarchTY * rr): D = A1 mz(0) + A2 kz(0)
    const T mdx = md_of(ax, i), kdx = kd_of(ax, i);
    T mdy[kMarchRows], kdy[kMarchRows], A1[kMarchRows], A2[kMarchRows], iDb[kMarchRows],
        iDi[kMarchRows];
    bool own[kMarchRows], exy[kMarchRows];
    int64_t off[kMarchRows];
#pragma unroll
    for (int rr = 0; rr < kMarchRows; ++rr) {
        const int j = j0 + ty + kMarchTY * rr;
        own[rr] = i < L.NX1 && j < L.NY1;
        mdy[rr] = md_of(ay, j);
        kdy[rr] = kd_of(ay, j);
        A1[rr] = kdx * mdy[rr] + mdx * kdy[rr] + L.kappa * mdx * mdy[rr];
        A2[rr] = mdx * mdy[rr];
        iDb[rr] = T(1) / (A1[rr] * az.m_bd + A2[rr] * az.k_bd);
        iDi[rr] = T(1) / (A1[rr] * az.m_in + A2[rr] * az.k_in);
        exy[rr] = (L.faces[0] && i == 0) || (L.faces[1] && i == L.NX1 - 1) ||
                  (L.faces[2] && j == 0) || (L.faces[3] && j == L.NY1 - 1);
        off[rr] = i + (int64_t)L.NX1 * j;
    }
    const int klast = min(k0 + M.kz, L.NZ1);  // planes k0 .. klast-1 are output
    auto stage = [&](int kk, T (&v)[kStagePer]) {
        const bool zcut = kk < 0 || kk >= L.NZ1 || (L.faces[4] && kk == 0) ||
                          (L.faces[5] && kk == L.NZ1 - 1);
        if constexpr (VX == kVb) {
            const bool zb = kk == 0 || kk == L.NZ1 - 1;
#pragma unroll
            for (int r = 0; r < kStagePer; ++r)
                v[r] = (s_in[r] && !zcut) ? M.inv_theta * M.b[s_off[r] + plane_n * kk] *
                                                (zb ? s_iDb[r] : s_iDi[r])
                                          : T(0);
        } else {
#pragma unroll
            for (int r = 0; r < kStagePer; ++r)
                v[r] = (s_in[r] && !zcut) ? vsrc<T, VX>(M, s_off[r] + plane_n * kk) : T(0);
        }
    };
    // per row: (P, Q) of planes k-1, k; the node inputs of the next output
    // plane (b, d, v) loaded one plane ahead, the staged planes two ahead
    T Pm[kMarchRows], P0[kMarchRows], Qm[kMarchRows], Q0[kMarchRows];
    T b_nx[kMarchRows], d_nx[kMarchRows], v_nx[kMarchRows];
#pragma unroll
    for (int rr = 0; rr < kMarchRows; ++rr)
        Pm[rr] = P0[rr] = Qm[rr] = Q0[rr] = b_nx[rr] = d_nx[rr] = v_nx[rr] = T(0);
    auto plane = [&](int kk, T (&cur)[kStagePer]) {
#pragma unroll
        for (int r = 0; r < kStagePer; ++r)
            if (tid + r * kMarchThreads < kStage) vt[tid + r * kMarchThreads] = cur[r];
        __syncthreads();
        T b_cur[kMarchRows], d_cur[kMarchRows], v_cur[kMarchRows];
#pragma unroll
        for (int rr = 0; rr < kMarchRows; ++rr) {
            b_cur[rr] = b_nx[rr];
            d_cur[rr] = d_nx[rr];
            v_cur[rr] = v_nx[rr];
        }
        // the loads two planes ahead are in flight while this plane is folded
        if (kk + 2 <= klast) stage(kk + 2, cur);
        const bool ez = (L.faces[4] && kk == 0) || (L.faces[5] && kk == L.NZ1 - 1);
        if (kk >= k0 && kk < klast) {
#pragma unroll
            for (int rr = 0; rr < kMarchRows; ++rr)
                if (own[rr]) {
                    const int64_t nd = off[rr] + plane_n * kk;
                    if (M.b) b_nx[rr] = M.b[nd];
                    if constexpr (VX == kVb) {
                        // v = d0 at the node (staged, unless eliminated)
                        const bool zb = kk == 0 || kk == L.NZ1 - 1;
                        v_nx[rr] = (exy[rr] || ez)
                                       ? M.inv_theta * b_nx[rr] * (zb ? iDb[rr] : iDi[rr])
                                       : vt[(ty + kMarchTY * rr + 1) * (kMarchX + 2) + tx + 1];
                        d_nx[rr] = v_nx[rr];
                    } else {
                        if (MODE == kMarchStep) d_nx[rr] = M.d[nd];
                        // v at the node: staged, unless eliminated (staged as 0)
                        v_nx[rr] = (exy[rr] || ez)
                                       ? vsrc<T, VX>(M, nd)
                                       : vt[(ty + kMarchTY * rr + 1) * (kMarchX + 2) + tx + 1];
                    }
                }
        }
        // the x rows of the plane at the CTA's columns, rows j0-1 .. j0+kMarchY
#pragma unroll
        for (int r = 0; r < kXRowPer; ++r) {
            const int q = tid + r * kMarchThreads;
            if (q < kXRows) {
                const T vm = vt[x_v[r]], v0 = vt[x_v[r] + 1], vp = vt[x_v[r] + 2];
                T a = T(0), c = T(0);
                a += ax.k_off * vm;
                c += ax.m_off * vm;
                a += x_k[r] * v0;
                c += x_m[r] * v0;
                a += ax.k_off * vp;
                c += ax.m_off * vp;
                sk[q] = a;
                sm[q] = c;
            }
        }
        __syncthreads();
        const int k = kk - 1;  // output plane: k-1, k, k+1 = (Pm, P0, Pp)
        const bool out = k >= k0 && k < klast;
        const bool bd = k == 0 || k == L.NZ1 - 1;
        const bool elim_z = (L.faces[4] && k == 0) || (L.faces[5] && k == L.NZ1 - 1);
        const T mdz = bd ? az.m_bd : az.m_in, kdz = bd ? az.k_bd : az.k_in;
#pragma unroll
        for (int rr = 0; rr < kMarchRows; ++rr) {
            // y fold for this row's column on plane kk
            const int c0 = (ty + kMarchTY * rr) * kMarchX + tx;
            T Ax = T(0), By = T(0), C = T(0);
            Ax += sk[c0] * ay.m_off;
            By += sm[c0] * ay.k_off;
            C += sm[c0] * ay.m_off;
            Ax += sk[c0 + kMarchX] * mdy[rr];
            By += sm[c0 + kMarchX] * kdy[rr];
            C += sm[c0 + kMarchX] * mdy[rr];
            Ax += sk[c0 + 2 * kMarchX] * ay.m_off;
            By += sm[c0 + 2 * kMarchX] * ay.k_off;
            C += sm[c0 + 2 * kMarchX] * ay.m_off;
            const T Pp = Ax + By + L.kappa * C, Qp = C;
            if (out && own[rr]) {
                const int64_t node = off[rr] + plane_n * k;
                T Av = T(0);
                Av += Pm[rr] * az.m_off;
                Av += Qm[rr] * az.k_off;
                Av += P0[rr] * mdz;
                Av += Q0[rr] * kdz;
                Av += Pp * az.m_off;
                Av += Qp * az.k_off;
                const T inv_D = bd ? iDb[rr] : iDi[rr];
                if (exy[rr] || elim_z) Av = (A1[rr] * mdz + A2[rr] * kdz) * v_cur[rr];
                if constexpr (MODE == kMarchApply) {
                    M.y[node] = M.b ? b_cur[rr] - Av : Av;
                } else if constexpr (MODE == kMarchCheb0) {
                    // first Chebyshev direction from x (not null here)
                    const T d0 = M.inv_theta * (b_cur[rr] - Av) * inv_D;
                    if (M.x_final)
                        M.x_final[node] = v_cur[rr] + d0;
                    else
                        M.d_next[node] = d0;
                } else {
                    const T dn = M.c1 * d_cur[rr] + M.c2 * ((b_cur[rr] - Av) * inv_D);
                    if (M.z4) {
                        M.z4[4 * node + 3] = (M.m4 && M.m4[4 * node + 3])
                                                 ? M.v4[4 * node + 3]
                                                 : (v_cur[rr] + dn) * M.inv_sigma;
                    } else if (M.x_final) {
                        M.x_final[node] = v_cur[rr] + dn;
                    } else {
                        M.x_next[node] = v_cur[rr];
                        M.d_next[node] = dn;
                    }
                }
            }
            Pm[rr] = P0[rr];
            Qm[rr] = Q0[rr];
            P0[rr] = Pp;
            Q0[rr] = Qp;
        }
        __syncthreads();
    };
    T pa[kStagePer], pb[kStagePer];
    stage(k0 - 1, pa);
    stage(k0, pb);
    for (int kk = k0 - 1; kk <= klast; kk += 2) {
        plane(kk, pa);
        if (kk + 1 <= klast) plane(kk + 1, pb);
    }
}

const dim3 kMarchBlock(kMarchX, kMarchTY);

template <typename T, int MODE, int VX>
fsi_status march_launch(const PressureMG &P, int l, cudaStream_t s, March<T> M)
{
    const PmgLevel &L = P.lev[l];
    const int nz1 = L.N[2] + 1;
    const int gx = (L.N[0] + 1 + kMarchX - 1) / kMarchX, gy = (L.N[1] + 1 + kMarchY - 1) / kMarchY;
    // planes per CTA: about 8 CTAs per SM in all (each CTA's planes are a
    // serial chain of shared-memory passes), at least 2, at most 16
    const int64_t cols = (int64_t)gx * gy;
    M.kz = (int)std::max<int64_t>(2, std::min<int64_t>(16, nz1 * cols / (16 * sm_count())));
    const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((nz1 + M.kz - 1) / M.kz));
    march_kernel<T, MODE, VX><<<grid, kMarchBlock, 0, s>>>(level_args<T>(P, l), M);
    return check_launch("pressure stencil");
}

// the stencil pass in MODE: on v = M.x (apply, first Chebyshev direction) or
// v = M.x + M.d (Chebyshev step; M.x null after a zero start; both null: the
// first step from x = 0, v = d0 = b / (theta D) formed in the pass)
template <typename T, int MODE>
fsi_status march(const PressureMG &P, int l, cudaStream_t s, const March<T> &M)
{
    if constexpr (MODE == kMarchStep) {
        if (M.x) return march_launch<T, MODE, kVxd>(P, l, s, M);
        if (M.d) return march_launch<T, MODE, kVd>(P, l, s, M);
        if (!M.b) return FSI_ERR_ARG;
        return march_launch<T, MODE, kVb>(P, l, s, M);  // the first step from x = 0
    } else {
        if (!M.x) return FSI_ERR_ARG;
        return march_launch<T, MODE, kVx>(P, l, s, M);
    }
}

// y = A x (b == null) or y = b - A x on level l
template <typename T>
fsi_status level_apply(const PressureMG &P, int l, cudaStream_t s, const T *x, const T *b, T *y)
{
    March<T> M{};
    M.x = x;
    M.b = b;
    M.y = y;
    return march<T, kMarchApply>(P, l, s, M);
}

// b_c = P^T r: each coarse node gathers the fine nodes within one fine cell,
// weights 1 (coincident) and 1/2 (neighbour) per axis; zero on eliminated nodes
template <typename T>
__global__ void restrict_kernel(LevelArgs<T> F, LevelArgs<T> C, const T *__restrict__ r,
                                T *__restrict__ bc)
{
    NODE3(C, I, J, K)
    {
        const int64_t node = I + (int64_t)C.NX1 * (J + (int64_t)C.NY1 * K);
        T acc = T(0);
        for (int dk = -1; dk <= 1; ++dk) {
            const int k = 2 * K + dk;
            if (k < 0 || k >= F.NZ1) continue;
            const T wk = dk ? T(0.5) : T(1);
            for (int dj = -1; dj <= 1; ++dj) {
                const int j = 2 * J + dj;
                if (j < 0 || j >= F.NY1) continue;
                const T wjk = (dj ? T(0.5) : T(1)) * wk;
                const T *row = r + (int64_t)F.NX1 * (j + (int64_t)F.NY1 * k);
                T s = T(0);
                for (int di = -1; di <= 1; ++di) {
                    const int i = 2 * I + di;
                    if (i < 0 || i >= F.NX1) continue;
                    s += (di ? T(0.5) : T(1)) * row[i];
                }
                acc += wjk * s;
            }
        }
        bc[node] = eliminated(C, I, J, K) ? T(0) : acc;
    }
}

// x += P x_c: trilinear interpolation of the coarse correction
template <typename T>
__global__ void prolong_kernel(LevelArgs<T> F, LevelArgs<T> C, const T *__restrict__ xc,
                               T *__restrict__ x)
{
    NODE3(F, i, j, k)
    {
        const int64_t node = i + (int64_t)F.NX1 * (j + (int64_t)F.NY1 * k);
        const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
        const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
        const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1),
                wk = (k & 1) ? T(0.5) : T(1);
        T acc = T(0);
        for (int c = 0; c < nk; ++c)
            for (int bb = 0; bb < nj; ++bb) {
                const T *row = xc + (int64_t)C.NX1 * ((j0 + bb) + (int64_t)C.NY1 * (k0 + c));
                T s = T(0);
                for (int a = 0; a < ni; ++a) s += row[i0 + a];
                acc += (wj * wk) * (wi * s);
            }
        x[node] += acc;
    }
}

template <typename T> __global__ void copy_kernel(int64_t n, const T *a, T *b)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        b[q] = a[q];
}

// x = Ainv b on the coarsest grid: one warp per row, fixed reduction order
template <typename T>
__global__ void dense_apply_kernel(int64_t nc, const T *__restrict__ Ainv, const T *__restrict__ b,
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

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 16)); }

// node kernels: CTAs of 32 nodes along x by 4 along y (at 129 nodes per row:
// 81 % of the lanes busy, against 50 % for 128-node rows of CTAs), one plane
// per grid layer
const dim3 kRowBlock(32, 4);
dim3 grid3(const PmgLevel &L)
{
    return dim3((unsigned)((L.N[0] + 1 + 31) / 32), (unsigned)((L.N[1] + 1 + 3) / 4),
                (unsigned)(L.N[2] + 1));
}
// the same with about 16 CTAs per SM in all, each striding over planes (for
// the purely pointwise first smoother direction: 13 -> 8 us at 129^3; the
// transfers are faster one plane per CTA)
dim3 grid3_strided(const PmgLevel &L)
{
    const int gx = (L.N[0] + 1 + 31) / 32, gy = (L.N[1] + 1 + 3) / 4;
    const int64_t gz = std::max<int64_t>(1, std::min<int64_t>(L.N[2] + 1,
                                                              16 * sm_count() / ((int64_t)gx * gy)));
    return dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
}

double spectrum_bound(const double h[3], double kappa)
{
    double diag = kappa;
    for (int d = 0; d < 3; ++d) diag *= 2.0 * h[d] / 3.0;
    for (int d = 0; d < 3; ++d) {
        double t = 2.0 / h[d];
        for (int e = 0; e < 3; ++e)
            if (e != d) t *= 2.0 * h[e] / 3.0;
        diag += t;
    }
    double best = 0.0;
    for (int s = 0; s < 8; ++s) {
        double k[3], m[3];
        for (int d = 0; d < 3; ++d) {
            const bool pi = (s >> d) & 1;
            k[d] = pi ? 4.0 / h[d] : 0.0;
            m[d] = pi ? h[d] / 3.0 : h[d];
        }
        const double sym = k[0] * m[1] * m[2] + m[0] * k[1] * m[2] + m[0] * m[1] * k[2] +
                           kappa * m[0] * m[1] * m[2];
        best = std::max(best, sym / diag);
    }
    return 1.1 * best;
}

// Dense K + kappa M of a (small) level from the same 1D coefficients, then
// its inverse by Gauss-Jordan with partial pivoting (FP64, host).
bool dense_inverse(const PmgLevel &L, double kappa, const int faces[6], std::vector<double> &inv)
{
    auto elim = [&](int i, int j, int k) {
        return (faces[0] && i == 0) || (faces[1] && i == L.N[0]) || (faces[2] && j == 0) ||
               (faces[3] && j == L.N[1]) || (faces[4] && k == 0) || (faces[5] && k == L.N[2]);
    };
    const int nx = L.N[0] + 1, ny = L.N[1] + 1, nz = L.N[2] + 1;
    const int64_t n = L.n;
    auto c1 = [&](int d, int i, int off, double &m, double &k) {
        const double h = L.h[d];
        if (off == 0) {
            const bool bd = i == 0 || i == L.N[d];
            m = bd ? h / 3.0 : 2.0 * h / 3.0;
            k = bd ? 1.0 / h : 2.0 / h;
        } else {
            m = h / 6.0;
            k = -1.0 / h;
        }
    };
    std::vector<double> a((size_t)n * 2 * n, 0.0);
    const int64_t w = 2 * n;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t row = i + (int64_t)nx * (j + (int64_t)ny * k);
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            const int ii = i + di, jj = j + dj, kk = k + dk;
                            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz)
                                continue;
                            double mx, kx, my, ky, mz, kz;
                            c1(0, i, di, mx, kx);
                            c1(1, j, dj, my, ky);
                            c1(2, k, dk, mz, kz);
                            const int64_t col = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
                            if (col != row && (elim(i, j, k) || elim(ii, jj, kk))) continue;
                            a[row * w + col] = kx * my * mz + mx * ky * mz + mx * my * kz +
                                               kappa * mx * my * mz;
                        }
                a[row * w + n + row] = 1.0;
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

template <typename T> T *vec(void *p) { return static_cast<T *>(p); }

// Chebyshev semi-iteration of `degree` on level l for A x = b over [lo, hi],
// from x_in (null: zero) into x_out; x_out may equal x_in only for degree 1.
// One kernel per step: step k reads (x_{k-1}, d_{k-1}) and writes
// (x_k, d_k) to the other buffers of a ping-pong pair; the last step writes
// x_m = x_{m-1} + d_{m-1} straight into x_out.
// the Schur preconditioner's output of the V-cycle (see March::z4)
template <typename T> struct SchurOut {
    T *z4;
    const T *v4;
    const uint8_t *m4;
    T inv_sigma;
};

template <typename T>
fsi_status chebyshev(fsi_mesh *m, int l, int degree, double lo, double hi, const T *b,
                     const T *x_in, T *x_out, const SchurOut<T> *so = nullptr)
{
    PressureMG &P = *m->pmg;
    PmgLevel &L = P.lev[l];
    const LevelArgs<T> A = level_args<T>(P, l);
    cudaStream_t s = m->stream;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), s1 = theta / delta;
    T *dbuf[2] = {vec<T>(L.d0), vec<T>(L.d1)}, *xbuf[2] = {vec<T>(L.xa), vec<T>(L.r)};
    // first direction (degree 1: x_out = x + d0 directly)
    if (x_in) {
        March<T> M{};
        M.x = x_in;
        M.b = b;
        M.inv_theta = (T)(1.0 / theta);
        M.d_next = degree == 1 ? nullptr : dbuf[0];
        M.x_final = degree == 1 ? x_out : nullptr;
        FSI_TRY((march<T, kMarchCheb0>(P, l, s, M)));
    } else if (degree == 1) {
        cheb0_kernel<T><<<grid3_strided(L), kRowBlock, 0, s>>>(A, b, (T)(1.0 / theta), nullptr,
                                                               x_out);
        FSI_TRY(check_launch("pressure smoother"));
    }
    if (degree == 1) return FSI_OK;
    // from x = 0 the first step forms d0 = b / (theta D) itself (no d0 pass)
    const T *xc = x_in;
    const T *dc = x_in ? dbuf[0] : nullptr;
    double rho = 1.0 / s1;
    for (int it = 1; it < degree; ++it) {
        const double rho_new = 1.0 / (2.0 * s1 - rho);
        const T c1 = (T)(rho_new * rho), c2 = (T)(2.0 * rho_new / delta);
        const bool last = it == degree - 1;
        T *xn = xbuf[it & 1], *dn = dbuf[it & 1];
        March<T> M{};
        M.x = xc;
        M.d = dc;
        M.b = b;
        M.c1 = c1;
        M.c2 = c2;
        M.inv_theta = (T)(1.0 / theta);
        M.x_next = last ? nullptr : xn;
        M.d_next = last ? nullptr : dn;
        M.x_final = last ? x_out : nullptr;
        if (last && so) {
            M.z4 = so->z4;
            M.v4 = so->v4;
            M.m4 = so->m4;
            M.inv_sigma = so->inv_sigma;
        }
        FSI_TRY((march<T, kMarchStep>(P, l, s, M)));
        xc = xn;
        dc = dn;
        rho = rho_new;
    }
    return check_launch("pressure smoother");
}

template <typename T> fsi_status coarse_solve(fsi_mesh *m, const T *b, T *x)
{
    PressureMG &P = *m->pmg;
    const int l = P.nlev - 1;
    if (P.direct) {
        const T *inv = std::is_same<T, double>::value ? (const T *)P.inv64 : (const T *)P.inv32;
        const int warps_per_block = 8;
        const int blocks = (int)std::min<int64_t>((P.nc + warps_per_block - 1) / warps_per_block, sm_count() * 8);
        dense_apply_kernel<T><<<blocks, 32 * warps_per_block, 0, m->stream>>>(P.nc, inv, b, x);
        return check_launch("pressure coarse solve");
    }
    return chebyshev<T>(m, l, kPmgCoarseDegree, P.lev[l].hi / 30.0, P.lev[l].hi, b, nullptr, x);
}

// x = V_l(b): pre-smoothing from zero into t, residual, restriction, the
// coarse cycle, prolongation into t, post-smoothing from t into x
// (so: level l's result goes to the Schur preconditioner's output instead of
// x; not on the coarsest level)
template <typename T>
fsi_status vcycle_level(fsi_mesh *m, int l, const T *b, T *x, const SchurOut<T> *so = nullptr)
{
    PressureMG &P = *m->pmg;
    if (l == P.nlev - 1) return coarse_solve<T>(m, b, x);
    PmgLevel &L = P.lev[l], &Lc = P.lev[l + 1];
    const double hi = L.hi;
    T *t = vec<T>(L.t);
    FSI_TRY(chebyshev<T>(m, l, kPmgNu, hi / 4.0, hi, b, (const T *)nullptr, t));
    const LevelArgs<T> A = level_args<T>(P, l), Ac = level_args<T>(P, l + 1);
    FSI_TRY(level_apply<T>(P, l, m->stream, t, b, vec<T>(L.r)));
    restrict_kernel<T><<<grid3(Lc), kRowBlock, 0, m->stream>>>(A, Ac, vec<T>(L.r), vec<T>(Lc.b));
    FSI_TRY(check_launch("pressure restrict"));
    FSI_TRY(vcycle_level<T>(m, l + 1, vec<T>(Lc.b), vec<T>(Lc.x)));
    prolong_kernel<T><<<grid3(L), kRowBlock, 0, m->stream>>>(A, Ac, vec<T>(Lc.x), t);
    FSI_TRY(check_launch("pressure prolong"));
    return chebyshev<T>(m, l, kPmgNu, hi / 4.0, hi, b, t, x, so);
}

fsi_status check_prec(fsi_prec p)
{
    if (p != FSI_F64 && p != FSI_F32) return set_error(FSI_ERR_ARG, "pressure operator: precision must be FSI_F64 or FSI_F32");
    return FSI_OK;
}

fsi_status check_level(fsi_mesh *m, int level, bool need_coarser)
{
    if (level < 0 || level >= m->pmg->nlev || (need_coarser && level + 1 >= m->pmg->nlev))
        return set_error(FSI_ERR_ARG, "pressure operator: level %d out of range", level);
    return FSI_OK;
}

}  // namespace

void destroy_pmg(fsi_mesh *m)
{
    if (!m->pmg) return;
    PressureMG &P = *m->pmg;
    for (int l = 0; l < P.nlev; ++l) {
        void *bufs[] = {P.lev[l].b, P.lev[l].x, P.lev[l].r, P.lev[l].t,
                        P.lev[l].d0, P.lev[l].d1, P.lev[l].xa};
        for (void *q : bufs) cudaFree(q);
    }
    cudaFree(P.inv64);
    cudaFree(P.inv32);
    delete m->pmg;
    m->pmg = nullptr;
}

// dense inverse of the coarsest level for the current faces (FP64 host
// Gauss-Jordan), copied to the device in FP64 and FP32
fsi_status build_coarse_inverse(fsi_mesh *m)
{
    PressureMG &P = *m->pmg;
    const PmgLevel &C = P.lev[P.nlev - 1];
    std::vector<double> inv;
    if (!dense_inverse(C, P.kappa, P.faces, inv))
        return set_error(FSI_ERR_ARG, "pressure hierarchy: singular coarse operator");
    std::vector<float> inv32(inv.begin(), inv.end());
    FSI_CUDA(cudaMemcpy(P.inv64, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice),
             "memcpy");
    FSI_CUDA(cudaMemcpy(P.inv32, inv32.data(), inv32.size() * sizeof(float),
                        cudaMemcpyHostToDevice),
             "memcpy");
    return FSI_OK;
}

fsi_status pmg_ensure(fsi_mesh *m)
{
    FSI_TRY(require_structured(m, "the pressure multigrid"));
    if (m->pmg) return FSI_OK;
    PressureMG *P = new (std::nothrow) PressureMG();
    if (!P) return set_error(FSI_ERR_OOM, "host allocation of the pressure hierarchy failed");
    m->pmg = P;
    double Lmax = 0.0;
    for (int d = 0; d < 3; ++d) Lmax = std::max(Lmax, m->grid.N[d] * m->grid.h[d]);
    const double q = 3.14159265358979323846 / (2.0 * Lmax);
    P->kappa = q * q;
    if (m->grid.N[1] + 1 > 65535 || m->grid.N[2] + 1 > 65535) {
        destroy_pmg(m);
        return set_error(FSI_ERR_ARG, "pressure hierarchy: at most 65535 nodes along y and z");
    }
    PmgLevel cur{};
    for (int d = 0; d < 3; ++d) {
        cur.N[d] = m->grid.N[d];
        cur.h[d] = m->grid.h[d];
    }
    while (true) {
        cur.n = (int64_t)(cur.N[0] + 1) * (cur.N[1] + 1) * (cur.N[2] + 1);
        cur.hi = spectrum_bound(cur.h, P->kappa);
        P->lev[P->nlev++] = cur;
        const bool even = cur.N[0] % 2 == 0 && cur.N[1] % 2 == 0 && cur.N[2] % 2 == 0;
        if (!even || cur.n <= kPmgMinCoarsen || P->nlev == kPmgMaxLevels) break;
        for (int d = 0; d < 3; ++d) {
            cur.N[d] /= 2;
            cur.h[d] *= 2.0;
        }
    }
    for (int l = 0; l < P->nlev; ++l) {
        const size_t bytes = (size_t)P->lev[l].n * sizeof(double);
        void **bufs[] = {&P->lev[l].b,  &P->lev[l].x,  &P->lev[l].r, &P->lev[l].t,
                         &P->lev[l].d0, &P->lev[l].d1, &P->lev[l].xa};
        for (void **b : bufs) {
            *b = nullptr;
            if (cudaMalloc(b, bytes) != cudaSuccess) {
                cudaGetLastError();
                destroy_pmg(m);
                return set_error(FSI_ERR_OOM, "pressure hierarchy: cudaMalloc failed");
            }
        }
    }
    const PmgLevel &C = P->lev[P->nlev - 1];
    P->nc = C.n;
    P->direct = C.n <= kPmgDirectMax;
    if (P->direct) {
        if (cudaMalloc((void **)&P->inv64, (size_t)C.n * C.n * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&P->inv32, (size_t)C.n * C.n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            destroy_pmg(m);
            return set_error(FSI_ERR_OOM, "pressure hierarchy: cudaMalloc failed");
        }
        fsi_status st = build_coarse_inverse(m);
        if (st != FSI_OK) {
            destroy_pmg(m);
            return st;
        }
    }
    return FSI_OK;
}

fsi_status pmg_set_faces(fsi_mesh *m, const int faces[6])
{
    FSI_TRY(pmg_ensure(m));
    PressureMG &P = *m->pmg;
    bool same = true;
    for (int f = 0; f < 6; ++f) same = same && (P.faces[f] != 0) == (faces[f] != 0);
    if (same) return FSI_OK;
    for (int f = 0; f < 6; ++f) P.faces[f] = faces[f] != 0;
    // the coarse inverse is in use by work already queued on the stream
    FSI_CUDA(cudaStreamSynchronize(m->stream), "sync");
    return P.direct ? build_coarse_inverse(m) : FSI_OK;
}

template <typename T> fsi_status pmg_vcycle(fsi_mesh *m, const T *b, T *x)
{
    FSI_TRY(pmg_ensure(m));
    return vcycle_level<T>(m, 0, b, x);
}
template fsi_status pmg_vcycle<double>(fsi_mesh *, const double *, double *);
template fsi_status pmg_vcycle<float>(fsi_mesh *, const float *, float *);

template <typename T>
fsi_status pmg_vcycle_schur(fsi_mesh *m, const T *b, T *z, const T *v, const uint8_t *mask,
                            T inv_sigma, bool *done)
{
    FSI_TRY(pmg_ensure(m));
    *done = false;
    PressureMG &P = *m->pmg;
    if (P.nlev < 2) return FSI_OK;
    const SchurOut<T> so{z, v, mask, inv_sigma};
    FSI_TRY(vcycle_level<T>(m, 0, b, vec<T>(P.lev[0].x), &so));
    *done = true;
    return FSI_OK;
}
template fsi_status pmg_vcycle_schur<double>(fsi_mesh *, const double *, double *, const double *,
                                             const uint8_t *, double, bool *);
template fsi_status pmg_vcycle_schur<float>(fsi_mesh *, const float *, float *, const float *,
                                            const uint8_t *, float, bool *);

// level-0 right-hand side (which = 0) and solution (which = 1) buffers, n
// entries of either precision; the Newton preconditioner gathers into them
void *pmg_fine_buffer(fsi_mesh *m, int which) { return which == 0 ? m->pmg->lev[0].b : m->pmg->lev[0].x; }

}  // namespace fsi

// ---------------------------------------------------------------- C ABI
using namespace fsi;

extern "C" {

fsi_status fsi_pressure_levels(fsi_mesh *mesh, int32_t *n_levels, int32_t *N)
{
    FSI_TRY(validate_mesh(mesh));
    if (!n_levels) return set_error(FSI_ERR_ARG, "fsi_pressure_levels: n_levels is NULL");
    if (mesh->pressure_amg)
        return set_error(FSI_ERR_ARG, "fsi_pressure_levels: the pressure block is the algebraic "
                                      "multigrid (fsi_pressure_level_sizes)");
    FSI_DEVICE(mesh->device);
    FSI_TRY(pmg_ensure(mesh));
    *n_levels = mesh->pmg->nlev;
    if (N)
        for (int l = 0; l < mesh->pmg->nlev; ++l)
            for (int d = 0; d < 3; ++d) N[3 * l + d] = mesh->pmg->lev[l].N[d];
    return FSI_OK;
}

fsi_status fsi_pressure_level_sizes(fsi_mesh *mesh, int32_t *n_levels, int64_t *n)
{
    FSI_TRY(validate_mesh(mesh));
    if (!n_levels) return set_error(FSI_ERR_ARG, "fsi_pressure_level_sizes: n_levels is NULL");
    FSI_DEVICE(mesh->device);
    if (uses_amg(mesh)) return amg_level_sizes(mesh, n_levels, n);
    FSI_TRY(pmg_ensure(mesh));
    *n_levels = mesh->pmg->nlev;
    if (n)
        for (int l = 0; l < mesh->pmg->nlev; ++l) n[l] = mesh->pmg->lev[l].n;
    return FSI_OK;
}

fsi_status fsi_pressure_set_eliminated(fsi_mesh *mesh, const uint8_t *eliminated)
{
    FSI_TRY(validate_mesh(mesh));
    if (!uses_amg(mesh))
        return set_error(FSI_ERR_ARG, "fsi_pressure_set_eliminated: the pressure block is the "
                                      "geometric multigrid (it eliminates faces: "
                                      "fsi_pressure_set_faces; or fsi_pressure_use_amg)");
    FSI_DEVICE(mesh->device);
    std::vector<uint8_t> e((size_t)mesh->n_nodes, 0);
    if (eliminated) {
        FSI_CUDA(cudaMemcpyAsync(e.data(), eliminated, e.size(), cudaMemcpyDeviceToHost,
                                 mesh->stream),
                 "memcpy");
        FSI_CUDA(cudaStreamSynchronize(mesh->stream), "sync");
        for (uint8_t &v : e) v = v != 0;
    }
    return amg_set_eliminated(mesh, e);
}

fsi_status fsi_pressure_use_amg(fsi_mesh *mesh, int32_t on)
{
    FSI_TRY(validate_mesh(mesh));
    if (mesh->tet) {
        if (!on)
            return set_error(FSI_ERR_ARG, "fsi_pressure_use_amg: a tetrahedral mesh has only the "
                                          "algebraic multigrid");
        return FSI_OK;
    }
    FSI_DEVICE(mesh->device);
    if ((on != 0) == mesh->pressure_amg) return FSI_OK;
    // the hierarchy may be in use by work already queued on the stream
    FSI_CUDA(cudaStreamSynchronize(mesh->stream), "sync");
    destroy_amg(mesh);
    mesh->pressure_amg = on != 0;
    return FSI_OK;
}

fsi_status fsi_pressure_set_faces(fsi_mesh *mesh, const int32_t *faces)
{
    FSI_TRY(validate_mesh(mesh));
    if (!faces) return set_error(FSI_ERR_ARG, "fsi_pressure_set_faces: faces is NULL");
    if (mesh->pressure_amg)
        return set_error(FSI_ERR_ARG, "fsi_pressure_set_faces: the pressure block is the "
                                      "algebraic multigrid (fsi_pressure_set_eliminated)");
    FSI_DEVICE(mesh->device);
    int f[6];
    for (int q = 0; q < 6; ++q) f[q] = faces[q] != 0;
    return pmg_set_faces(mesh, f);
}

fsi_status fsi_pressure_apply(fsi_mesh *mesh, fsi_prec prec, int32_t level, const void *x, void *y)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(check_prec(prec));
    if (!x || !y) return set_error(FSI_ERR_ARG, "fsi_pressure_apply: NULL argument");
    FSI_DEVICE(mesh->device);
    if (uses_amg(mesh)) return amg_apply(mesh, prec, level, x, y);
    FSI_TRY(pmg_ensure(mesh));
    FSI_TRY(check_level(mesh, level, false));
    if (prec == FSI_F64)
        return level_apply<double>(*mesh->pmg, level, mesh->stream, (const double *)x, nullptr,
                                   (double *)y);
    return level_apply<float>(*mesh->pmg, level, mesh->stream, (const float *)x, nullptr,
                              (float *)y);
}

fsi_status fsi_pressure_restrict(fsi_mesh *mesh, fsi_prec prec, int32_t level, const void *r,
                                 void *b)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(check_prec(prec));
    if (!r || !b) return set_error(FSI_ERR_ARG, "fsi_pressure_restrict: NULL argument");
    FSI_DEVICE(mesh->device);
    if (uses_amg(mesh)) return amg_restrict(mesh, prec, level, r, b);
    FSI_TRY(pmg_ensure(mesh));
    FSI_TRY(check_level(mesh, level, true));
    PressureMG &P = *mesh->pmg;
    const dim3 g = grid3(P.lev[level + 1]);
    if (prec == FSI_F64)
        restrict_kernel<double><<<g, kRowBlock, 0, mesh->stream>>>(
            level_args<double>(P, level), level_args<double>(P, level + 1), (const double *)r,
            (double *)b);
    else
        restrict_kernel<float><<<g, kRowBlock, 0, mesh->stream>>>(
            level_args<float>(P, level), level_args<float>(P, level + 1), (const float *)r,
            (float *)b);
    return check_launch("pressure restrict");
}

fsi_status fsi_pressure_prolong_add(fsi_mesh *mesh, fsi_prec prec, int32_t level,
                                    const void *xc, void *x)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(check_prec(prec));
    if (!xc || !x) return set_error(FSI_ERR_ARG, "fsi_pressure_prolong_add: NULL argument");
    FSI_DEVICE(mesh->device);
    if (uses_amg(mesh)) return amg_prolong_add(mesh, prec, level, xc, x);
    FSI_TRY(pmg_ensure(mesh));
    FSI_TRY(check_level(mesh, level, true));
    PressureMG &P = *mesh->pmg;
    const dim3 g = grid3(P.lev[level]);
    if (prec == FSI_F64)
        prolong_kernel<double><<<g, kRowBlock, 0, mesh->stream>>>(
            level_args<double>(P, level), level_args<double>(P, level + 1), (const double *)xc,
            (double *)x);
    else
        prolong_kernel<float><<<g, kRowBlock, 0, mesh->stream>>>(
            level_args<float>(P, level), level_args<float>(P, level + 1), (const float *)xc,
            (float *)x);
    return check_launch("pressure prolong");
}

fsi_status fsi_pressure_smooth(fsi_mesh *mesh, fsi_prec prec, int32_t level, int32_t degree,
                               const void *b, void *x, int32_t from_zero)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(check_prec(prec));
    if (!b || !x) return set_error(FSI_ERR_ARG, "fsi_pressure_smooth: NULL argument");
    if (degree < 1 || degree > 64) return set_error(FSI_ERR_ARG, "fsi_pressure_smooth: degree 1..64");
    FSI_DEVICE(mesh->device);
    if (uses_amg(mesh)) return amg_smooth(mesh, prec, level, degree, b, x, from_zero);
    FSI_TRY(pmg_ensure(mesh));
    FSI_TRY(check_level(mesh, level, false));
    const double hi = mesh->pmg->lev[level].hi;
    const int64_t n = mesh->pmg->lev[level].n;
    // from a given x: the iteration reads x while it writes the result, so
    // it starts from a copy in the level's t buffer
    if (prec == FSI_F64) {
        const double *xin = nullptr;
        if (!from_zero) {
            copy_kernel<double><<<grid_for(n), 256, 0, mesh->stream>>>(
                n, (const double *)x, (double *)mesh->pmg->lev[level].t);
            xin = (const double *)mesh->pmg->lev[level].t;
        }
        return chebyshev<double>(mesh, level, degree, hi / 4.0, hi, (const double *)b, xin,
                                 (double *)x);
    }
    const float *xin = nullptr;
    if (!from_zero) {
        copy_kernel<float><<<grid_for(n), 256, 0, mesh->stream>>>(
            n, (const float *)x, (float *)mesh->pmg->lev[level].t);
        xin = (const float *)mesh->pmg->lev[level].t;
    }
    return chebyshev<float>(mesh, level, degree, hi / 4.0, hi, (const float *)b, xin, (float *)x);
}

fsi_status fsi_pressure_vcycle(fsi_mesh *mesh, fsi_prec prec, const void *b, void *x)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(check_prec(prec));
    if (!b || !x) return set_error(FSI_ERR_ARG, "fsi_pressure_vcycle: NULL argument");
    if (b == x) return set_error(FSI_ERR_ARG, "fsi_pressure_vcycle: b and x must not alias");
    FSI_DEVICE(mesh->device);
    if (uses_amg(mesh)) {
        if (prec == FSI_F64) return amg_vcycle<double>(mesh, (const double *)b, (double *)x);
        return amg_vcycle<float>(mesh, (const float *)b, (float *)x);
    }
    if (prec == FSI_F64) return pmg_vcycle<double>(mesh, (const double *)b, (double *)x);
    return pmg_vcycle<float>(mesh, (const float *)b, (float *)x);
}

}  // extern "C"
