// dlm.cu -- fictitious-domain coupling operators (Sec. 2.3 of the paper):
// point location with a cell -> points table, interpolation u = C^T V
// (Eq. nodal_solid_velo) and spreading F = C lambda (Eq. fsi_constraint_matrix).
//
// Location is closed-form on the uniform grid (a bounded element walk with
// Newton inversion on a mapped grid).  The cell table is a stable counting
// sort: histogram (integer atomics, order-free), a three-kernel exclusive
// scan, a scatter through per-cell cursors, and a per-cell sort of each
// cell's slice by point index, which restores the stable order exactly (a
// bitonic network in one lane's registers up to 64 points, a warp rank sort
// up to 128, a shell sort beyond).  Spreading is atomic-free in two passes:
// per-cell corner sums (four lanes per cell of up to 128 points, the warp for
// fuller cells, fixed transpose-reduce trees), then a node gather over the
// (up to) eight cells of each node in a fixed order.  No races, no atomics,
// and the result does not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <mutex>

#include "fsi_internal.cuh"
#include "dlm_device.cuh"

namespace fsi {
namespace {

using namespace dlmd;

GridArgs grid_args(const fsi_mesh *m)
{
    GridArgs g;
    g.Nx = m->grid.N[0];
    g.Ny = m->grid.N[1];
    g.Nz = m->grid.N[2];
    g.x0 = m->grid.x0[0];
    g.y0 = m->grid.x0[1];
    g.z0 = m->grid.x0[2];
    g.hx = m->grid.h[0];
    g.hy = m->grid.h[1];
    g.hz = m->grid.h[2];
    set_reciprocals(g);
    return g;
}

int blocks_for(int64_t n, int threads, int cap = sm_count() * 16)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// grid of the node pass (32 x 8 CTAs over (i, j)): about 16 CTAs per SM in
// all, the z index striding over the planes (one plane per CTA made the CTA
// launches the limit at 2.1 M nodes)
dim3 node_grid(const GridArgs &g)
{
    const int gx = (g.Nx + 32) / 32, gy = std::min((g.Ny + 8) / 8, 65535);
    const int64_t gz = std::max<int64_t>(
        1, std::min<int64_t>(std::min(g.Nz + 1, 65535), 16 * sm_count() / ((int64_t)gx * gy)));
    return dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
}

// --------------------------------------------------------------- locate
__global__ void locate_kernel(int64_t m, GridArgs g, const double *__restrict__ X,
                              int32_t *__restrict__ elem, double *__restrict__ xi,
                              int32_t *__restrict__ count, unsigned long long *n_out)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int e = locate_point<double>(g, b, X, elem, xi);
        if (e < 0)
            atomicAdd(n_out, 1ull);
        else if (count)
            atomicAdd(count + e, 1);
    }
}

// Mapped grid (node coordinates C [n][4]): element walk guided by Newton's
// method on the trilinear map x(xi) = sum_a N_a(xi) x_a.
//
// Walk (FP32, coordinates relative to the element's first node): start in
// the element the nominal uniform box gives (clamped); solve x(xi) = X there
// (at most 16 iterations from xi = 0); the extended map's root tells how many
// elements away the point lies, so the first 6 moves jump floor((xi_k+1)/2)
// elements per axis (at most 8), later moves one element across the face of
// the largest violation.  Once the FP32 root lies in the cube widened by 1e-3,
// Newton's method in FP64 from that root decides: a settled root (last update
// below 1e-12) with |xi_k| <= 1 + 1e-10 places the point; otherwise the FP64
// root steers the next move.  At most Nx + Ny + Nz + 8 elements; leaving the
// grid, a singular map or running out of moves is "outside".  Every loop is
// bounded.
struct HexNodes {
    double o[3];      // first node
    double d[8][3];   // node - first node
};

__device__ __forceinline__ void load_hex(const GridArgs &g, const double4 *__restrict__ C, int ex,
                                         int ey, int ez, HexNodes &H)
{
    const int NX1 = g.Nx + 1, NXY1 = (g.Nx + 1) * (g.Ny + 1);
    const int64_t n0 = ex + (int64_t)NX1 * ey + (int64_t)NXY1 * ez;
    const double4 c0 = C[n0];
    H.o[0] = c0.x;
    H.o[1] = c0.y;
    H.o[2] = c0.z;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const double4 c = C[n0 + (a & 1) + NX1 * ((a >> 1) & 1) + (int64_t)NXY1 * ((a >> 2) & 1)];
        H.d[a][0] = c.x - c0.x;
        H.d[a][1] = c.y - c0.y;
        H.d[a][2] = c.z - c0.z;
    }
}

// One Newton update d of x(xi) = Y (Y relative to the first node): r, J at xi,
// J d = r by Cramer's rule.  False when J is singular.
template <typename R>
__device__ __forceinline__ bool newton_update(const R (&xa)[8][3], const R (&Y)[3], const R (&xi)[3],
                                              R (&d)[3])
{
    R r[3] = {-Y[0], -Y[1], -Y[2]}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const R s0 = (a & 1) ? R(1) : R(-1), s1 = (a & 2) ? R(1) : R(-1), s2 = (a & 4) ? R(1) : R(-1);
        const R l0 = R(1) + s0 * xi[0], l1 = R(1) + s1 * xi[1], l2 = R(1) + s2 * xi[2];
        const R N = R(0.125) * l0 * l1 * l2;
        const R d0 = R(0.125) * s0 * l1 * l2, d1 = R(0.125) * l0 * s1 * l2, d2 = R(0.125) * l0 * l1 * s2;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            r[i] += N * xa[a][i];
            J[i][0] += xa[a][i] * d0;
            J[i][1] += xa[a][i] * d1;
            J[i][2] += xa[a][i] * d2;
        }
    }
    const R c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const R c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const R c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const R det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(fabs(det) > R(0))) return false;
    const R inv = R(1) / det;
    d[0] = (r[0] * c00 + J[0][1] * (J[1][2] * r[2] - r[1] * J[2][2]) +
            J[0][2] * (r[1] * J[2][1] - J[1][1] * r[2])) * inv;
    d[1] = (J[0][0] * (r[1] * J[2][2] - J[1][2] * r[2]) + r[0] * c01 +
            J[0][2] * (J[1][0] * r[2] - r[1] * J[2][0])) * inv;
    d[2] = (J[0][0] * (J[1][1] * r[2] - r[1] * J[2][1]) +
            J[0][1] * (r[1] * J[2][0] - J[1][0] * r[2]) + r[0] * c02) * inv;
    return true;
}

// FP32 root of the extended map: 1 settled, 0 not settled (xi = last iterate,
// a direction only), -1 singular or blown up.
__device__ int newton_f32(const HexNodes &H, const double X[3], float (&xi)[3])
{
    float xa[8][3], Y[3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) xa[a][i] = (float)H.d[a][i];
#pragma unroll
    for (int i = 0; i < 3; ++i) Y[i] = (float)(X[i] - H.o[i]);
    xi[0] = xi[1] = xi[2] = 0.0f;
    for (int it = 0; it < 16; ++it) {
        float d[3];
        if (!newton_update<float>(xa, Y, xi, d)) return -1;
        xi[0] -= d[0];
        xi[1] -= d[1];
        xi[2] -= d[2];
        if (!(fabsf(xi[0]) < 64.0f && fabsf(xi[1]) < 64.0f && fabsf(xi[2]) < 64.0f)) return -1;
        if (fmaxf(fabsf(d[0]), fmaxf(fabsf(d[1]), fabsf(d[2]))) < 1e-5f) return 1;
    }
    return 0;
}

// FP64-accurate root from the start xi (the settled FP32 root): true when
// settled (last update < 1e-12).  The Newton updates run in double-float
// arithmetic on the FP32 pipe (~48-bit significands; GB300's FP64 unit is
// 1/64 of its FP32 rate and bounded the location kernel): node offsets and
// X - o are formed in FP64 (one rounding) and split exactly to 2^-47, so the
// root agrees with an FP64 Newton iteration to ~1e-14 in xi.  The start is
// within ~1e-7 of the root, so the second update is ~1e-14: the loop stops
// once an update is below 1e-13.
__device__ bool newton_df(const HexNodes &H, const double X[3], double (&xi)[3])
{
    df64 xa[8][3], Y[3], q[3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) xa[a][i] = df_split(H.d[a][i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Y[i] = df_split(X[i] - H.o[i]);
        q[i] = df_split(xi[i]);
    }
    const df64 one(1), eighth(0.125f);
    float last = 1.0f;
    for (int it = 0; it < 12; ++it) {
        df64 r[3] = {-Y[0], -Y[1], -Y[2]}, J[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) J[i][0] = J[i][1] = J[i][2] = df64(0);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const df64 l0 = (a & 1) ? one + q[0] : one - q[0];
            const df64 l1 = (a & 2) ? one + q[1] : one - q[1];
            const df64 l2 = (a & 4) ? one + q[2] : one - q[2];
            const df64 l12 = l1 * l2, l01 = l0 * l1, l02 = l0 * l2;
            // N and dN/dxi_k, the factor 1/8 and the signs are exact
            const df64 N = eighth * (l0 * l12);
            const df64 d0 = (a & 1) ? eighth * l12 : -(eighth * l12);
            const df64 d1 = (a & 2) ? eighth * l02 : -(eighth * l02);
            const df64 d2 = (a & 4) ? eighth * l01 : -(eighth * l01);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                r[i] = df_fma(N, xa[a][i], r[i]);
                J[i][0] = df_fma(xa[a][i], d0, J[i][0]);
                J[i][1] = df_fma(xa[a][i], d1, J[i][1]);
                J[i][2] = df_fma(xa[a][i], d2, J[i][2]);
            }
        }
        const df64 c00 = df_dot2(J[1][1], J[2][2], -J[1][2], J[2][1]);
        const df64 c01 = df_dot2(J[1][2], J[2][0], -J[1][0], J[2][2]);
        const df64 c02 = df_dot2(J[1][0], J[2][1], -J[1][1], J[2][0]);
        const df64 det = df_fma(J[0][2], c02, df_dot2(J[0][0], c00, J[0][1], c01));
        if (!(fabsf(det.hi) > 0.0f)) return false;
        const df64 inv = df_rcp(det);
        // Cramer's rule: the same cofactor expansion as the FP64 update
        const df64 n0 = df_fma(J[0][2], df_dot2(r[1], J[2][1], -J[1][1], r[2]),
                               df_dot2(r[0], c00, J[0][1], df_dot2(J[1][2], r[2], -r[1], J[2][2])));
        const df64 n1 = df_fma(J[0][2], df_dot2(J[1][0], r[2], -r[1], J[2][0]),
                               df_dot2(J[0][0], df_dot2(r[1], J[2][2], -J[1][2], r[2]), r[0], c01));
        const df64 n2 = df_fma(r[0], c02, df_dot2(J[0][0], df_dot2(J[1][1], r[2], -r[1], J[2][1]),
                                                  J[0][1], df_dot2(r[1], J[2][0], -J[1][0], r[2])));
        const df64 d[3] = {n0 * inv, n1 * inv, n2 * inv};
#pragma unroll
        for (int i = 0; i < 3; ++i) q[i] = q[i] - d[i];
        if (!(fabsf(q[0].hi) < 64.0f && fabsf(q[1].hi) < 64.0f && fabsf(q[2].hi) < 64.0f))
            return false;
        last = fmaxf(fabsf(d[0].hi), fmaxf(fabsf(d[1].hi), fabsf(d[2].hi)));
        if (last < 1e-13f) break;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) xi[i] = q[i].to_double();
    return last < 1e-12f;
}

__global__ void locate_mapped_kernel(int64_t m, GridArgs g, const double4 *__restrict__ C,
                                     const double *__restrict__ Xp, int32_t *__restrict__ elem,
                                     double *__restrict__ xi, int32_t *__restrict__ count,
                                     unsigned long long *n_out)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const double X[3] = {Xp[3 * b], Xp[3 * b + 1], Xp[3 * b + 2]};
        const double t[3] = {(X[0] - g.x0) / g.hx, (X[1] - g.y0) / g.hy, (X[2] - g.z0) / g.hz};
        const int N3[3] = {g.Nx, g.Ny, g.Nz};
        int e3[3];
        bool finite = true;
        for (int k = 0; k < 3; ++k) {
            finite = finite && isfinite(t[k]) && isfinite(X[k]);
            const double c = finite ? floor(t[k]) : 0.0;
            e3[k] = c < 0.0 ? 0 : (c > (double)(N3[k] - 1) ? N3[k] - 1 : (int)c);
        }
        int found = 0;
        double q[3] = {0.0, 0.0, 0.0};
        const int max_steps = g.Nx + g.Ny + g.Nz + 8;
        for (int step = 0; step < max_steps && finite; ++step) {
            HexNodes H;
            load_hex(g, C, e3[0], e3[1], e3[2], H);
            float q32[3];
            const int st = newton_f32(H, X, q32);
            // direction of the next move, from the FP64 root where there is one
            double dir[3] = {q32[0], q32[1], q32[2]};
            bool jump = st == 1 && step < 6;
            if (st == 1 && fabsf(q32[0]) <= 1.001f && fabsf(q32[1]) <= 1.001f &&
                fabsf(q32[2]) <= 1.001f) {
                q[0] = q32[0];
                q[1] = q32[1];
                q[2] = q32[2];
                const bool ok = newton_df(H, X, q);
                if (ok && fabs(q[0]) <= 1.0 + 1e-10 && fabs(q[1]) <= 1.0 + 1e-10 &&
                    fabs(q[2]) <= 1.0 + 1e-10) {
                    found = 1;
                    break;
                }
                if (!ok) break;
                dir[0] = q[0];
                dir[1] = q[1];
                dir[2] = q[2];
                jump = false;
            }
            if (st < 0) break;
            if (jump) {
                bool moved = false;
                for (int k = 0; k < 3; ++k) {
                    double s = floor(0.5 * (dir[k] + 1.0));
                    s = s > 8.0 ? 8.0 : (s < -8.0 ? -8.0 : s);
                    int nk = e3[k] + (int)s;
                    nk = nk < 0 ? 0 : (nk > N3[k] - 1 ? N3[k] - 1 : nk);
                    moved = moved || nk != e3[k];
                    e3[k] = nk;
                }
                if (moved) continue;
                // clamped at the grid's edge: fall through to a plain move
            }
            int k = 0;
            double worst = fabs(dir[0]);
            for (int d = 1; d < 3; ++d)
                if (fabs(dir[d]) > worst) {
                    worst = fabs(dir[d]);
                    k = d;
                }
            if (!(worst > 1.0)) break;
            const int next = e3[k] + (dir[k] > 0.0 ? 1 : -1);
            if (next < 0 || next >= N3[k]) break;
            e3[k] = next;
        }
        if (!found) {
            elem[b] = -1;
            xi[3 * b] = xi[3 * b + 1] = xi[3 * b + 2] = 0.0;
            atomicAdd(n_out, 1ull);
            continue;
        }
        const int e = e3[0] + g.Nx * (e3[1] + g.Ny * e3[2]);
        elem[b] = e;
        xi[3 * b] = q[0];
        xi[3 * b + 1] = q[1];
        xi[3 * b + 2] = q[2];
        if (count) atomicAdd(count + e, 1);
    }
}

// --------------------------------------------------------------- cell table
// (the per-work-item bodies are in dlm_device.cuh, shared with the batch)
__global__ void __launch_bounds__(1024) scan_tiles_kernel(int64_t E, const int32_t *count,
                                                          int32_t *start, int32_t *tile_sum)
{
    __shared__ int warp_sums[32];
    scan_tile(E, count, start, tile_sum, blockIdx.x, warp_sums);
}

__global__ void __launch_bounds__(1024) scan_totals_kernel(int64_t ntiles, int32_t *tile_sum)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    scan_totals_block(ntiles, tile_sum, warp_sums, &carry);
}

__global__ void scan_add_kernel(int64_t E, int32_t *start, const int32_t *tile_sum)
{
    scan_add_tile(E, start, tile_sum, blockIdx.x);
}

__global__ void scatter_kernel(int64_t m, int64_t E, const int32_t *__restrict__ elem,
                               const int32_t *__restrict__ start, int32_t *fill,
                               int32_t *__restrict__ perm)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x)
        scatter_point(b, E, elem, start, fill, perm);
}

__global__ void cell_sort_kernel(int64_t E, int64_t m, const int32_t *__restrict__ start,
                                 int32_t *__restrict__ perm, int32_t *dense, int32_t *dense_count)
{
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c0 = warp * 32; c0 <= E; c0 += nwarps * 32)
        cell_sort_segment(E, m, start, perm, c0, dense, dense_count);
}

// the cells listed by cell_sort_kernel, one CTA per cell
__global__ void __launch_bounds__(1024) dense_sort_kernel(int64_t E, int64_t m,
                                                          const int32_t *__restrict__ start,
                                                          int32_t *__restrict__ perm,
                                                          const int32_t *dense,
                                                          const int32_t *dense_count)
{
    extern __shared__ int32_t sort_sh[];
    const int n = *dense_count;
    for (int k = blockIdx.x; k < n; k += gridDim.x)
        block_sort_cell(E, m, start, perm, dense[k], sort_sh);
}

// --------------------------------------------------------------- interp / spread
// FP32: two lanes per point (interp_point_pair; the loop bound is
// warp-uniform); double-float and FP64: one lane per point
template <typename T, typename S = typename StorageOf<T>::type>
__global__ void interp_kernel(int64_t m, GridArgs g, const int32_t *__restrict__ elem,
                              const S *__restrict__ xi, const vec4<S> *__restrict__ U,
                              S *__restrict__ u)
{
    if constexpr (std::is_same<T, float>::value) {
        const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        const int pair = (threadIdx.x & 31) >> 1;
        for (int64_t b0 = warp * 16; b0 < m; b0 += nwarps * 16)
            interp_point_pair<T>(g, b0 + pair, b0 + pair < m, elem, xi, U, u);
    } else {
        for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
             b += (int64_t)gridDim.x * blockDim.x)
            interp_point<T>(g, b, elem, xi, U, u);
    }
}

// Spreading, pass 1: one warp per segment of kSpreadSeg consecutive cells
// (see spread_cells_segment).
// T is the compute type (double, float or double-float); xi, lam, w and F are
// in its storage type, the corner sums S in T.
// (SQ: w N^2 dsq instead of w N lambda, see spread_accumulate)
template <typename T, bool SQ = false>
__global__ void spread_cells_kernel(int64_t E, const typename StorageOf<T>::type *__restrict__ xi,
                                    const int32_t *__restrict__ start,
                                    const int32_t *__restrict__ perm,
                                    const typename StorageOf<T>::type *__restrict__ lam,
                                    const typename StorageOf<T>::type *__restrict__ w,
                                    T *__restrict__ S, T dsq = T(0))
{
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c0 = warp * kSpreadSeg; c0 < E; c0 += nwarps * kSpreadSeg)
        spread_cells_segment<T, SQ>(E, c0, xi, start, perm, lam, w, S, dsq);
}

// Spreading, pass 2: every node sums the corner sums of its occupied cells.
// 3D launch: x over the row's nodes, y over j, z (strided) over k: no index
// division.
template <typename T>
__global__ void spread_nodes_kernel(GridArgs g, const int32_t *__restrict__ start,
                                    const T *__restrict__ S,
                                    typename StorageOf<T>::type *__restrict__ F, int accumulate)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.Nx || j > g.Ny) return;
    for (int k = blockIdx.z; k <= g.Nz; k += gridDim.z)
        spread_node<T>(g, i, j, k, start, S, F, accumulate);
}

// ------------------------------------------------------------- interface scaling
// s at node (i, j, k) = s_band when one of the cells within `layers` cells of
// the node's (up to) 8 cells holds a point, 1 otherwise: the node touches a
// band cell exactly when a cell of [i-1-layers, i+layers] x ... (clipped) is
// occupied.
__global__ void interface_scaling_kernel(int Nx, int Ny, int Nz, const int32_t *__restrict__ start,
                                         double s_band, int layers, double *__restrict__ s)
{
    const int NX1 = Nx + 1, NY1 = Ny + 1;
    const int64_t n = (int64_t)NX1 * NY1 * (Nz + 1);
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < n;
         node += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(node % NX1), j = (int)((node / NX1) % NY1),
                  k = (int)(node / ((int64_t)NX1 * NY1));
        const int i0 = max(0, i - 1 - layers), i1 = min(Nx - 1, i + layers);
        const int j0 = max(0, j - 1 - layers), j1 = min(Ny - 1, j + layers);
        const int k0 = max(0, k - 1 - layers), k1 = min(Nz - 1, k + layers);
        bool on = false;
        for (int c = k0; c <= k1 && !on; ++c)
            for (int b = j0; b <= j1 && !on; ++b) {
                const int64_t row = (int64_t)Nx * (b + (int64_t)Ny * c);
                for (int a = i0; a <= i1; ++a)
                    if (start[row + a + 1] > start[row + a]) {
                        on = true;
                        break;
                    }
            }
        s[node] = on ? s_band : 1.0;
    }
}

// ---------------------------------------------------------------- no-allocation locate
// fsi_locate_noalloc keeps its scratch (outside-point counter, per-cell fill
// counters, scan tile sums) in one file-scope device array instead of mesh
// memory, so it never allocates.  Layout in int32 slots: [0, 64) counter
// (first 8 bytes), [64, 64 + kNoAllocMaxCells + 1 rounded up) fill counters,
// then the tile sums.  About 16 MB per device, held until the process exits.
constexpr int64_t kNoAllocMaxCells = 4000000;
constexpr int64_t kNoAllocFillOffset = 64;
constexpr int64_t kNoAllocTileOffset =
    kNoAllocFillOffset + ((kNoAllocMaxCells + 1 + 63) / 64) * 64;
constexpr int64_t kNoAllocInts =
    kNoAllocTileOffset + ((kNoAllocMaxCells + kScanTile - 1) / kScanTile + 64);
static __device__ __align__(256) int32_t g_locate_scratch[kNoAllocInts];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
int32_t *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_locate_scratch on `device` (which must be current),
// looked up once per device.  Host code cannot use the symbol itself: its
// host-side name is only a stand-in, not a device address.
fsi_status noalloc_scratch(int device, int32_t **out)
{
    if (device < 0 || device >= kNoAllocMaxDevices)
        return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        FSI_CUDA(cudaGetSymbolAddress(&p, g_locate_scratch),
                 "fsi_locate_noalloc: cudaGetSymbolAddress of the static scratch");
        g_noalloc_addr[device] = (int32_t *)p;
    }
    *out = g_noalloc_addr[device];
    return FSI_OK;
}

GridArgs grid_args_of(const fsi_grid &gr)
{
    GridArgs g;
    g.Nx = gr.N[0];
    g.Ny = gr.N[1];
    g.Nz = gr.N[2];
    g.x0 = gr.x0[0];
    g.y0 = gr.x0[1];
    g.z0 = gr.x0[2];
    g.hx = gr.h[0];
    g.hy = gr.h[1];
    g.hz = gr.h[2];
    set_reciprocals(g);
    return g;
}

}  // namespace

// the scan's tile sums and, after them, the count of CTA-sorted cells
int64_t cell_table_scan_ints(int64_t E) { return cell_tiles(E) + 1; }

fsi_status build_cell_table(cudaStream_t s, int64_t E, int64_t m, const int32_t *elem,
                            int32_t *fill, int32_t *scan_tmp, int32_t *cell_start, int32_t *perm)
{
    const int64_t ntiles = cell_tiles(E);
    scan_tiles_kernel<<<(int)ntiles, 1024, 0, s>>>(E, fill, cell_start, scan_tmp);
    FSI_TRY(check_launch("scan tiles kernel"));
    scan_totals_kernel<<<1, 1024, 0, s>>>(ntiles, scan_tmp);
    FSI_TRY(check_launch("scan totals kernel"));
    scan_add_kernel<<<(int)ntiles, 256, 0, s>>>(E, cell_start, scan_tmp);
    FSI_TRY(check_launch("scan add kernel"));
    if (m > 0) {
        FSI_CUDA(cudaMemsetAsync(fill, 0, (E + 1) * sizeof(int32_t), s), "memset");
        scatter_kernel<<<blocks_for(m, 256), 256, 0, s>>>(m, E, elem, cell_start, fill, perm);
        FSI_TRY(check_launch("scatter kernel"));
        // the cursors in fill are spent: fill lists the cells too full for a
        // warp, scan_tmp[ntiles] counts them
        int32_t *dense_count = scan_tmp + ntiles;
        FSI_CUDA(cudaMemsetAsync(dense_count, 0, sizeof(int32_t), s), "memset");
        cell_sort_kernel<<<blocks_for((E + 32) / 32 * 32, 256, sm_count() * 64), 256, 0, s>>>(
            E, m, cell_start, perm, fill, dense_count);
        FSI_TRY(check_launch("cell sort kernel"));
        if (m > kWarpSortMax) {
            const int smem = kBlockSortMax * (int)sizeof(int32_t);
            FSI_TRY(set_smem_limit((const void *)dense_sort_kernel, smem));
            dense_sort_kernel<<<sm_count(), 1024, smem, s>>>(E, m, cell_start, perm, fill,
                                                            dense_count);
            FSI_TRY(check_launch("dense cell sort kernel"));
        }
    }
    return FSI_OK;
}

template <typename T>
fsi_status spread_mass_diag(fsi_mesh *mesh, int64_t m, const T *xi, const int32_t *cell_start,
                            const int32_t *perm, const T *w, double dsq, T *F)
{
    (void)m;  // the cell table lists the points
    FSI_DEVICE(mesh->device);
    const GridArgs g = grid_args(mesh);
    const int64_t E = mesh->n_elems;
    FSI_TRY(ensure_spread_scratch(mesh, (size_t)E * 24 * sizeof(T)));
    const int cgrid = blocks_for((E + kSpreadSeg - 1) / kSpreadSeg * 32, 256, sm_count() * 64);
    spread_cells_kernel<T, true><<<cgrid, 256, 0, mesh->stream>>>(
        E, xi, cell_start, perm, nullptr, w, (T *)mesh->spread_scratch, (T)dsq);
    FSI_TRY(check_launch("spread cells kernel"));
    const dim3 nblock(32, 8), ngrid = node_grid(g);
    if ((g.Ny + 8) / 8 > 65535)
        return set_error(FSI_ERR_ARG, "spreading: more than 524,280 nodes along y");
    spread_nodes_kernel<T><<<ngrid, nblock, 0, mesh->stream>>>(g, cell_start,
                                                              (const T *)mesh->spread_scratch, F, 0);
    return check_launch("spread nodes kernel");
}
template fsi_status spread_mass_diag<float>(fsi_mesh *, int64_t, const float *, const int32_t *,
                                            const int32_t *, const float *, double, float *);
template fsi_status spread_mass_diag<double>(fsi_mesh *, int64_t, const double *,
                                             const int32_t *, const int32_t *, const double *,
                                             double, double *);

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status fsi_locate(fsi_mesh *mesh, int64_t m, const double *X, int32_t *elem, double *xi,
                      int32_t *cell_start, int32_t *perm, int64_t *n_outside, int strict)
{
    FSI_TRY(validate_mesh(mesh));
    if (m < 0 || m >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_locate: m out of range");
    if (m > 0 && (!X || !elem || !xi))
        return set_error(FSI_ERR_ARG, "fsi_locate: NULL X, elem or xi");
    if (perm != nullptr && cell_start == nullptr)
        return set_error(FSI_ERR_ARG, "fsi_locate: perm given without cell_start");
    if (cell_start != nullptr && perm == nullptr && m > 0)
        return set_error(FSI_ERR_ARG, "fsi_locate: cell_start given without perm");
    FSI_DEVICE(mesh->device);
    if (mesh->tet) {
        int64_t h = 0;
        FSI_TRY(fsi_tet_locate(mesh->tet, m, X, elem, xi, cell_start, perm,
                               (n_outside || strict) ? &h : nullptr));
        if (n_outside) *n_outside = h;
        if (strict && h > 0)
            return set_error(FSI_ERR_OUTSIDE, "fsi_locate: %lld points outside the mesh",
                             (long long)h);
        return FSI_OK;
    }
    const int64_t E = mesh->n_elems;
    cudaStream_t s = mesh->stream;
    unsigned long long *nout = (unsigned long long *)mesh->dev_counters;
    FSI_CUDA(cudaMemsetAsync(nout, 0, sizeof(unsigned long long), s), "memset");
    const bool table = cell_start != nullptr;
    if (table) FSI_CUDA(cudaMemsetAsync(mesh->hash_fill, 0, (E + 1) * sizeof(int32_t), s), "memset");
    GridArgs g = grid_args(mesh);
    if (m > 0 && mesh->coords64) {
        locate_mapped_kernel<<<blocks_for(m, 128), 128, 0, s>>>(
            m, g, (const double4 *)mesh->coords64, X, elem, xi,
            table ? mesh->hash_fill : nullptr, nout);
        FSI_TRY(check_launch("locate kernel"));
    } else if (m > 0) {
        locate_kernel<<<blocks_for(m, 256), 256, 0, s>>>(m, g, X, elem, xi,
                                                         table ? mesh->hash_fill : nullptr, nout);
        FSI_TRY(check_launch("locate kernel"));
    }
    if (table)
        FSI_TRY(build_cell_table(s, E, m, elem, mesh->hash_fill, mesh->scan_tmp, cell_start, perm));
    if (n_outside || strict) {
        unsigned long long h = 0;
        FSI_CUDA(cudaMemcpyAsync(&h, nout, sizeof h, cudaMemcpyDeviceToHost, s), "memcpy");
        FSI_CUDA(cudaStreamSynchronize(s), "stream sync");
        if (n_outside) *n_outside = (int64_t)h;
        if (strict && h > 0)
            return set_error(FSI_ERR_OUTSIDE, "fsi_locate: %llu points outside the grid", h);
    }
    return FSI_OK;
}

fsi_status fsi_dlm_interp(fsi_mesh *mesh, fsi_prec prec, int64_t m, const int32_t *elem,
                          const void *xi, const void *U, void *u)
{
    FSI_TRY(validate_mesh(mesh));
    if (m < 0 || m >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_dlm_interp: m out of range");
    if (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "bad precision");
    if (m == 0) return FSI_OK;
    if (!elem || !xi || !U || !u) return set_error(FSI_ERR_ARG, "fsi_dlm_interp: NULL argument");
    FSI_DEVICE(mesh->device);
    if (mesh->tet) return fsi_tet_interp(mesh->tet, prec, m, elem, xi, U, u);
    GridArgs g = grid_args(mesh);
    if (prec == FSI_F64)
        interp_kernel<double><<<blocks_for(m, 256), 256, 0, mesh->stream>>>(
            m, g, elem, (const double *)xi, (const vec4<double> *)U, (double *)u);
    else if (prec == FSI_DF64)
        interp_kernel<df64><<<blocks_for(m, 256), 256, 0, mesh->stream>>>(
            m, g, elem, (const double *)xi, (const vec4<double> *)U, (double *)u);
    else
        interp_kernel<float><<<blocks_for(2 * m, 256), 256, 0, mesh->stream>>>(
            m, g, elem, (const float *)xi, (const vec4<float> *)U, (float *)u);
    return check_launch("interp kernel");
}

fsi_status fsi_dlm_spread(fsi_mesh *mesh, fsi_prec prec, int64_t m, const int32_t *elem,
                          const void *xi, const int32_t *cell_start, const int32_t *perm,
                          const void *lam, const void *w, void *F, int accumulate)
{
    (void)elem;
    FSI_TRY(validate_mesh(mesh));
    if (m < 0 || m >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_dlm_spread: m out of range");
    if (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "bad precision");
    if (!F || !cell_start) return set_error(FSI_ERR_ARG, "fsi_dlm_spread: NULL F or cell_start");
    if (m > 0 && (!xi || !perm || !lam))
        return set_error(FSI_ERR_ARG, "fsi_dlm_spread: NULL xi, perm or lam");
    FSI_DEVICE(mesh->device);
    if (mesh->tet)
        return fsi_tet_spread(mesh->tet, prec, m, elem, xi, cell_start, perm, lam, w, F,
                              accumulate);
    GridArgs g = grid_args(mesh);
    // corner sums: 8 bytes per value for FP64 and double-float, 4 for FP32
    const size_t esz = prec == FSI_F32 ? sizeof(float) : sizeof(double);
    FSI_TRY(ensure_spread_scratch(mesh, (size_t)mesh->n_elems * 24 * esz));
    const int64_t E = mesh->n_elems;
    const int cgrid = blocks_for((E + kSpreadSeg - 1) / kSpreadSeg * 32, 256, sm_count() * 64);
    // nodes: 32 x 8 threads per CTA over (i, j), one grid layer per k
    const dim3 nblock(32, 8), ngrid = node_grid(g);
    if ((g.Ny + 8) / 8 > 65535)
        return set_error(FSI_ERR_ARG, "fsi_dlm_spread: more than 524,280 nodes along y");
    if (prec == FSI_F64) {
        spread_cells_kernel<double><<<cgrid, 256, 0, mesh->stream>>>(
            E, (const double *)xi, cell_start, perm, (const double *)lam, (const double *)w,
            (double *)mesh->spread_scratch);
        FSI_TRY(check_launch("spread cells kernel"));
        spread_nodes_kernel<double><<<ngrid, nblock, 0, mesh->stream>>>(
            g, cell_start, (const double *)mesh->spread_scratch, (double *)F, accumulate);
    } else if (prec == FSI_DF64) {
        spread_cells_kernel<df64><<<cgrid, 256, 0, mesh->stream>>>(
            E, (const double *)xi, cell_start, perm, (const double *)lam, (const double *)w,
            (df64 *)mesh->spread_scratch);
        FSI_TRY(check_launch("spread cells kernel"));
        spread_nodes_kernel<df64><<<ngrid, nblock, 0, mesh->stream>>>(
            g, cell_start, (const df64 *)mesh->spread_scratch, (double *)F, accumulate);
    } else {
        spread_cells_kernel<float><<<cgrid, 256, 0, mesh->stream>>>(
            E, (const float *)xi, cell_start, perm, (const float *)lam, (const float *)w,
            (float *)mesh->spread_scratch);
        FSI_TRY(check_launch("spread cells kernel"));
        spread_nodes_kernel<float><<<ngrid, nblock, 0, mesh->stream>>>(
            g, cell_start, (const float *)mesh->spread_scratch, (float *)F, accumulate);
    }
    return check_launch("spread nodes kernel");
}

fsi_status fsi_interface_scaling(fsi_mesh *mesh, const int32_t *cell_start, double s_band,
                                 int32_t layers, double *s)
{
    if (mesh) FSI_TRY(require_structured(mesh, "fsi_interface_scaling"));
    FSI_TRY(validate_mesh(mesh));
    if (!cell_start || !s) return set_error(FSI_ERR_ARG, "fsi_interface_scaling: NULL argument");
    if (!(s_band > 0.0) || !std::isfinite(s_band))
        return set_error(FSI_ERR_ARG, "fsi_interface_scaling: s_band must be positive and finite");
    if (layers < 0 || layers > 64)
        return set_error(FSI_ERR_ARG, "fsi_interface_scaling: layers must be in [0, 64]");
    FSI_DEVICE(mesh->device);
    const fsi_grid &g = mesh->grid;
    interface_scaling_kernel<<<blocks_for(mesh->n_nodes, 256), 256, 0, mesh->stream>>>(
        g.N[0], g.N[1], g.N[2], cell_start, s_band, layers, s);
    return check_launch("interface scaling kernel");
}

fsi_status fsi_locate_noalloc(const fsi_grid *grid, int64_t m, const double *X, int32_t *elem,
                              double *xi, int32_t *cell_start, int32_t *perm, int64_t *n_outside,
                              int strict, int device, void *cuda_stream)
{
    if (!grid) return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: grid is NULL");
    // The cell count bounds every index into the static scratch, so it is
    // checked after each factor: a product of three large int32 extents
    // could otherwise wrap around and pass the limit.
    int64_t E = 1;
    for (int k = 0; k < 3; ++k) {
        if (grid->N[k] < 1 || !(grid->h[k] > 0.0) || !std::isfinite(grid->h[k]) ||
            !std::isfinite(grid->x0[k]))
            return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: invalid grid");
        if (grid->N[k] > kNoAllocMaxCells || E * grid->N[k] > kNoAllocMaxCells)
            return set_error(FSI_ERR_ARG,
                             "fsi_locate_noalloc: grid %d x %d x %d has more cells than the "
                             "static scratch maximum of %lld; use fsi_locate with a mesh instead",
                             grid->N[0], grid->N[1], grid->N[2], (long long)kNoAllocMaxCells);
        E *= grid->N[k];
    }
    if (m < 0 || m >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: m out of range");
    if (m > 0 && (!X || !elem || !xi))
        return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: NULL X, elem or xi");
    if (perm != nullptr && cell_start == nullptr)
        return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: perm given without cell_start");
    if (cell_start != nullptr && perm == nullptr && m > 0)
        return set_error(FSI_ERR_ARG, "fsi_locate_noalloc: cell_start given without perm");
    FSI_DEVICE(device);
    int32_t *scratch = nullptr;
    FSI_TRY(noalloc_scratch(device, &scratch));
    unsigned long long *nout = (unsigned long long *)scratch;
    int32_t *fill = scratch + kNoAllocFillOffset;
    int32_t *tiles = scratch + kNoAllocTileOffset;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: clear what must start at zero
    FSI_CUDA(cudaMemsetAsync(nout, 0, sizeof(unsigned long long), s), "memset");
    const bool table = cell_start != nullptr;
    if (table) FSI_CUDA(cudaMemsetAsync(fill, 0, (E + 1) * sizeof(int32_t), s), "memset");
    GridArgs g = grid_args_of(*grid);
    if (m > 0) {
        locate_kernel<<<blocks_for(m, 256), 256, 0, s>>>(m, g, X, elem, xi, table ? fill : nullptr,
                                                         nout);
        FSI_TRY(check_launch("locate kernel"));
    }
    if (table) FSI_TRY(build_cell_table(s, E, m, elem, fill, tiles, cell_start, perm));
    if (n_outside || strict) {
        unsigned long long h = 0;
        FSI_CUDA(cudaMemcpyAsync(&h, nout, sizeof h, cudaMemcpyDeviceToHost, s), "memcpy");
        FSI_CUDA(cudaStreamSynchronize(s), "stream sync");
        if (n_outside) *n_outside = (int64_t)h;
        if (strict && h > 0)
            return set_error(FSI_ERR_OUTSIDE, "fsi_locate_noalloc: %llu points outside the grid",
                             h);
    }
    return FSI_OK;
}

}  // extern "C"
