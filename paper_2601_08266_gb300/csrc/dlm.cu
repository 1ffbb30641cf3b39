// dlm.cu -- fictitious-domain coupling operators (Sec. 2.3 of the paper):
// point location with a cell -> points table, interpolation u = C^T V
// (Eq. nodal_solid_velo) and spreading F = C lambda (Eq. fsi_constraint_matrix).
//
// Location is closed-form on the uniform grid (integer work on the bits of
// the coordinates when the spacings are powers of two; a bounded element
// walk with Newton inversion on a mapped grid).  The cell table is a stable
// counting sort: histogram (integer atomics, order-free), a single-pass
// exclusive scan with decoupled look-back, a scatter that counts the
// per-cell counters back down, and a per-cell sort of each cell's slice by
// point index, which restores the stable order exactly (a warp rank sort up
// to 128 points, a CTA bitonic network or a shell sort beyond).  Spreading
// is atomic-free in two passes:
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
template <bool ZERO_ORIGIN>
__global__ void locate_kernel(int64_t m, GridArgs g, const double *__restrict__ X,
                              int32_t *__restrict__ elem, double *__restrict__ xi,
                              int32_t *__restrict__ count, unsigned long long *n_out,
                              int32_t *__restrict__ arrival);

fsi_status launch_locate(cudaStream_t s, int64_t m, const GridArgs &g, const double *X,
                         int32_t *elem, double *xi, int32_t *count, unsigned long long *n_out,
                         int32_t *arrival = nullptr)
{
    if (g.shifted && g.zero_origin)
        locate_kernel<true><<<blocks_for(m, 256), 256, 0, s>>>(m, g, X, elem, xi, count, n_out,
                                                               arrival);
    else
        locate_kernel<false><<<blocks_for(m, 256), 256, 0, s>>>(m, g, X, elem, xi, count, n_out,
                                                                arrival);
    return check_launch("locate kernel");
}

// One atomic per point: leaflet points arrive in no spatial order, so the
// points of a warp almost never share a cell (a __match_any_sync grouping
// measured no fewer atomics and kept the address unit busy).  With arrival,
// each point keeps the count its cell had before it (outside points count in
// the tail cell E): its slot in the cell's slice, so the scatter needs no
// atomics.
template <bool ZERO_ORIGIN>
__global__ void locate_kernel(int64_t m, GridArgs g, const double *__restrict__ X,
                              int32_t *__restrict__ elem, double *__restrict__ xi,
                              int32_t *__restrict__ count, unsigned long long *n_out,
                              int32_t *__restrict__ arrival)
{
    const int64_t E = (int64_t)g.Nx * g.Ny * g.Nz;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int e = locate_point<double, ZERO_ORIGIN>(g, b, X, elem, xi);
        if (arrival) {
            arrival[b] = atomicAdd(count + (e >= 0 ? (int64_t)e : E), 1);
        } else if (e < 0) {
            if (n_out) atomicAdd(n_out, 1ull);
        } else if (count) {
            atomicAdd(count + e, 1);
        }
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
                                     unsigned long long *n_out, int32_t *__restrict__ arrival)
{
    const int64_t E = (int64_t)g.Nx * g.Ny * g.Nz;
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
            if (n_out) atomicAdd(n_out, 1ull);
            if (arrival) arrival[b] = atomicAdd(count + E, 1);
            continue;
        }
        const int e = e3[0] + g.Nx * (e3[1] + g.Ny * e3[2]);
        elem[b] = e;
        xi[3 * b] = q[0];
        xi[3 * b + 1] = q[1];
        xi[3 * b + 2] = q[2];
        if (arrival)
            arrival[b] = atomicAdd(count + e, 1);
        else if (count)
            atomicAdd(count + e, 1);
    }
}

// --------------------------------------------------------------- cell table
// Launches, none of them a memset: (1) the counts come from the locate
// kernel; (2) per-tile sums of the counts (2048 cells a tile); (3) the scan
// proper: each tile adds up the sums of the tiles before it (read from L2;
// beyond kDirectTiles tiles one CTA first scans the tile sums in place, an
// extra launch) and scans its own cells into start; (4) a scatter that counts
// each cell's counter back down to zero while it hands out the cell's slots
// (outside points take slots of the tail from a cursor); (5) a sort of every
// 32-cell segment's slices by point index, which restores the stable order
// exactly; cells of more than kWarpSortMax points are listed and sorted by a
// whole CTA (6, only when m > kWarpSortMax).  No kernel waits on another CTA.
// The counters and the scratch are left all zero, so the next call starts
// without clearing them.
//
// Scan scratch, int32 words: [0] count of CTA-sorted cells, [5] cursor of
// the outside points, [1..5) and [6, 8) unused, then the tile sums.
constexpr int kScanHdr = 8;
constexpr int kLbThreads = 256, kLbPer = kScanTile / kLbThreads;
constexpr int64_t kDirectTiles = 1024;

// this thread's kLbPer counts of tile t (zero past E)
__device__ __forceinline__ void tile_counts(int64_t E, const int32_t *__restrict__ count, int t,
                                            int (&v)[kLbPer])
{
    const int64_t base = (int64_t)t * kScanTile + (int64_t)threadIdx.x * kLbPer;
    if (base + kLbPer <= E) {
        const int4 a = *(const int4 *)(count + base), c = *(const int4 *)(count + base + 4);
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = c.x, v[5] = c.y, v[6] = c.z,
        v[7] = c.w;
    } else {
#pragma unroll
        for (int i = 0; i < kLbPer; ++i) v[i] = base + i < E ? count[base + i] : 0;
    }
}

__device__ __forceinline__ int block_sum(int x, int *warp_sums)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();  // warp_sums may still be read by a previous call
    if (lane == 0) warp_sums[wid] = x;
    __syncthreads();
    int s = 0;
#pragma unroll
    for (int w = 0; w < kLbThreads / 32; ++w) s += warp_sums[w];
    return s;
}

__global__ void __launch_bounds__(kLbThreads) tile_sums_kernel(int64_t E,
                                                               const int32_t *__restrict__ count,
                                                               int32_t *__restrict__ tile_sum)
{
    __shared__ int warp_sums[kLbThreads / 32];
    int v[kLbPer];
    tile_counts(E, count, blockIdx.x, v);
    int own = 0;
#pragma unroll
    for (int i = 0; i < kLbPer; ++i) own += v[i];
    const int s = block_sum(own, warp_sums);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
}

// exclusive scan of the tile sums in place (one CTA; many tiles only)
__global__ void __launch_bounds__(1024) tile_prefix_kernel(int64_t ntiles, int32_t *tile_sum)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    scan_totals_block(ntiles, tile_sum, warp_sums, &carry);
}

// DIRECT: the tile's prefix is the sum of tile_sum[0, t); else tile_sum[t]
template <bool DIRECT>
__global__ void __launch_bounds__(kLbThreads) tile_scan_kernel(int64_t E,
                                                               const int32_t *__restrict__ count,
                                                               const int32_t *__restrict__ tile_sum,
                                                               int32_t *__restrict__ start)
{
    __shared__ int warp_sums[kLbThreads / 32];
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v[kLbPer];
    tile_counts(E, count, t, v);
    int prefix;
    if constexpr (DIRECT) {
        int p = 0;
        for (int u = threadIdx.x; u < t; u += kLbThreads) p += tile_sum[u];
        prefix = block_sum(p, warp_sums);
    } else {
        prefix = tile_sum[t];
    }
    int own = 0;
#pragma unroll
    for (int i = 0; i < kLbPer; ++i) own += v[i];
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int w = 0; w < kLbThreads / 32; ++w) before += w < wid ? warp_sums[w] : 0;
    int run = prefix + before + incl - own;
    // through shared memory (a row of kLbPer + 1 ints per thread: no bank
    // conflicts) to stores of consecutive cells by consecutive threads
    __shared__ int out[kLbThreads * (kLbPer + 1)];
#pragma unroll
    for (int i = 0; i < kLbPer; ++i) {
        run += v[i];
        out[threadIdx.x * (kLbPer + 1) + i] = run;
    }
    __syncthreads();
    const int64_t base = (int64_t)t * kScanTile;
#pragma unroll
    for (int i = 0; i < kLbPer; ++i) {
        const int c = threadIdx.x + kLbThreads * i;
        if (base + c < E) start[base + c + 1] = out[(c / kLbPer) * (kLbPer + 1) + c % kLbPer];
    }
    if (t == 0 && threadIdx.x == 0) start[0] = 0;
}

// point b into a slot of its cell's slice: the cell's counter counts down,
// outside points count the tail cursor up (a slot outside [0, m), impossible
// with counts from this call's locate, is dropped rather than written)
__global__ void scatter_down_kernel(int64_t m, int64_t E, const int32_t *__restrict__ elem,
                                    const int32_t *__restrict__ start, int32_t *fill,
                                    int32_t *scr, int32_t *__restrict__ perm)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) scr[0] = 0;  // the sort lists dense cells afresh
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int e = elem[b];
        const int64_t pos = e >= 0 ? (int64_t)start[e] + atomicSub(fill + e, 1) - 1
                                   : (int64_t)start[E] + atomicAdd(scr + 5, 1);
        if (pos >= 0 && pos < m) perm[pos] = (int32_t)b;
    }
}

// Sort the slices of the cells [c0, c0 + 32) (one warp).  The slices are
// contiguous in perm, [S0, S0 + T) with S0 = start[c0] (the tail cell E
// holds the outside points).  A segment of at most 32 points is sorted at
// once by the key (cell, point index): lane k holds element k, finds its
// cell by a binary search over the 32 slice starts held in the lanes, and
// its new place is the number of the segment's elements with a smaller key
// (the keys are distinct).  A segment of up to kSegStage points is staged in
// shared memory with one coalesced load, and its cells of 2 to kWarpSortMax
// points are rank-sorted from there one at a time (so no cell waits for a
// load of its own); cells of more points go to the dense list (or, without
// one, to a single-lane shell sort).  Fuller segments sort their cells from
// global memory.
constexpr int kSegStage = 512;

__device__ __forceinline__ void sort_segment_small(int32_t *__restrict__ perm, int S0, int T,
                                                   int lo)
{
    const int lane = threadIdx.x & 31;
    const int v = lane < T ? perm[S0 + lane] : INT32_MAX;
    int q = 0;  // the last lane whose slice starts at or before S0 + lane
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(0xffffffffu, lo, q + step) <= S0 + lane) q += step;
    const int cl = lane < T ? q : 32;
    int rk = 0;
    for (int j = 0; j < T; ++j) {
        const int vj = __shfl_sync(0xffffffffu, v, j);
        const int cj = __shfl_sync(0xffffffffu, cl, j);
        rk += (cj < cl) | ((cj == cl) & (vj < v));
    }
    __syncwarp();
    if (lane < T) perm[S0 + rk] = v;
}

// rank sort of one slice of n (2..kWarpSortMax) values read from src, written
// to dst (src may be dst: every value is read before the first write)
__device__ __forceinline__ void rank_sort_slice(const int32_t *src, int32_t *dst, int n)
{
    const int lane = threadIdx.x & 31;
    if (n <= 32) {
        const int v = lane < n ? src[lane] : INT32_MAX;
        int rk = 0;
        for (int j = 0; j < n; ++j) rk += __shfl_sync(0xffffffffu, v, j) < v;
        __syncwarp();
        if (lane < n) dst[rk] = v;
        return;
    }
    int own[4], rk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        own[k] = (lane + 32 * k < n) ? src[lane + 32 * k] : INT32_MAX;
        rk[k] = 0;
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int jn = min(32, n - 32 * cc);  // warp-uniform
        for (int j = 0; j < jn; ++j) {
            const int wj = __shfl_sync(0xffffffffu, own[cc], j);
#pragma unroll
            for (int k = 0; k < 4; ++k) rk[k] += wj < own[k];
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (lane + 32 * k < n) dst[rk[k]] = own[k];
}

__device__ __forceinline__ void cell_sort_warp(int64_t E, int64_t m,
                                               const int32_t *__restrict__ start,
                                               int32_t *__restrict__ perm, int64_t c0,
                                               int32_t *dense, int32_t *dense_count,
                                               int32_t *stage)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = c0 + lane;
    int lo = (int)m, len = 0;
    if (c <= E) {
        lo = start[c];
        len = (c < E ? start[c + 1] : (int)m) - lo;
    }
    const int S0 = __shfl_sync(0xffffffffu, lo, 0);
    const int T = __shfl_sync(0xffffffffu, lo + len, 31) - S0;
    if (!__any_sync(0xffffffffu, len >= 2)) return;
    if (T <= 32) {
        sort_segment_small(perm, S0, T, lo);
        return;
    }
    if (dense && len > kWarpSortMax) dense[atomicAdd(dense_count, 1)] = (int32_t)c;
    const bool staged = stage != nullptr && T <= kSegStage;
    if (staged) {
        for (int k = lane; k < T; k += 32) stage[k] = perm[S0 + k];
        __syncwarp();
    }
    unsigned todo = __ballot_sync(0xffffffffu, len >= 2 && (len <= kWarpSortMax || !dense));
    while (todo) {
        const int l = __ffs(todo) - 1;
        todo &= todo - 1;
        const int base = __shfl_sync(0xffffffffu, lo, l);
        const int n = __shfl_sync(0xffffffffu, len, l);
        if (n <= kWarpSortMax) {
            rank_sort_slice(staged ? stage + (base - S0) : perm + base, perm + base, n);
        } else {
            __syncwarp();
            if (lane == 0) shell_sort(perm + base, n);
        }
        __syncwarp();
    }
}

constexpr int kSortThreads = 256;

__global__ void __launch_bounds__(kSortThreads) cell_sort_kernel(int64_t E, int64_t m,
                                                                 const int32_t *__restrict__ start,
                                                                 int32_t *__restrict__ perm,
                                                                 int32_t *dense, int32_t *scr)
{
    __shared__ int32_t stage[kSortThreads / 32][kSegStage];
    if (blockIdx.x == 0 && threadIdx.x == 0) scr[5] = 0;  // the outside cursor is spent
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c0 = warp * 32; c0 <= E; c0 += nwarps * 32)
        cell_sort_warp(E, m, start, perm, c0, dense, scr, stage[threadIdx.x >> 5]);
}

// the cells listed by cell_sort_kernel, one CTA per cell; each list entry is
// cleared once its cell is sorted (the list lives in the zeroed counters)
__global__ void __launch_bounds__(1024) dense_sort_kernel(int64_t E, int64_t m,
                                                          const int32_t *__restrict__ start,
                                                          int32_t *__restrict__ perm,
                                                          int32_t *dense,
                                                          const int32_t *dense_count)
{
    extern __shared__ int32_t sort_sh[];
    const int n = *dense_count;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int c = dense[k];
        block_sort_cell(E, m, start, perm, c, sort_sh);  // ends with __syncthreads
        if (threadIdx.x == 0) dense[k] = 0;
    }
}

// With point scratch (the mesh path): the scatter writes (point, cell) pairs
// into tmp, and every slot finds its point's final place in one pass: the
// number of points of its cell's slice with a smaller index (reads of the
// slice hit L1: the lanes of a warp mostly share a cell).  Cells of more than
// kWarpSortMax points are listed (by their first slot) and sorted by a CTA
// from tmp into perm.
// the points into (point, cell) pairs at their arrival slots; the point
// that arrived first at a cell clears the cell's counter
__global__ void scatter_arrival_kernel(int64_t m, int64_t E, const int32_t *__restrict__ elem,
                                       const int32_t *__restrict__ arrival,
                                       const int32_t *__restrict__ start, int32_t *fill,
                                       int32_t *scr, int2 *__restrict__ tmp)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) scr[0] = 0;  // the dense list starts empty
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int e = elem[b];
        const int c = e >= 0 ? e : (int)E;
        const int r = arrival[b];
        const int64_t pos = (int64_t)start[c] + r;
        if (pos >= 0 && pos < m) tmp[pos] = make_int2((int)b, c);
        if (r == 0) fill[c] = 0;
    }
}

__global__ void rank_place_kernel(int64_t m, int64_t E, const int32_t *__restrict__ start,
                                  const int2 *__restrict__ tmp, int32_t *__restrict__ perm,
                                  int32_t *dense, int32_t *scr)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = tmp[k];
        const int lo = start[p.y];
        const int hi = p.y < E ? start[p.y + 1] : (int)m;
        if (hi - lo > kWarpSortMax) {
            if (k == lo) dense[atomicAdd(scr, 1)] = p.y;
            continue;
        }
        // two pairs per 16-byte load from an even slot on
        int r = 0, j = lo;
        if ((j & 1) && j < hi) r += tmp[j++].x < p.x;
#pragma unroll 2
        for (; j + 1 < hi; j += 2) {
            const int4 q = *reinterpret_cast<const int4 *>(tmp + j);
            r += (q.x < p.x) + (q.z < p.x);
        }
        if (j < hi) r += tmp[j].x < p.x;
        perm[lo + r] = p.x;
    }
}

// the listed cells, one CTA per cell, from tmp into perm (bitonic network
// in shared memory, or one lane's shell sort beyond kBlockSortMax points);
// each list entry is cleared once its cell is sorted
__global__ void __launch_bounds__(1024) dense_pairs_kernel(int64_t E, int64_t m,
                                                           const int32_t *__restrict__ start,
                                                           const int2 *__restrict__ tmp,
                                                           int32_t *__restrict__ perm,
                                                           int32_t *dense,
                                                           const int32_t *dense_count)
{
    extern __shared__ int32_t sort_sh[];
    const int n = *dense_count;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int c = dense[k];
        const int lo = start[c];
        const int len = (c < E ? start[c + 1] : (int)m) - lo;
        for (int i = threadIdx.x; i < len; i += blockDim.x) perm[lo + i] = tmp[lo + i].x;
        __syncthreads();
        block_sort_cell(E, m, start, perm, c, sort_sh);  // ends with __syncthreads
        if (threadIdx.x == 0) dense[k] = 0;
    }
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
    kNoAllocTileOffset + kScanHdr + ((kNoAllocMaxCells + kScanTile - 1) / kScanTile) + 64;
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

// the scan's header and the tile sums (see the cell table)
int64_t cell_table_scan_ints(int64_t E) { return kScanHdr + cell_tiles(E) + 8; }

fsi_status build_cell_table(cudaStream_t s, int64_t E, int64_t m, const int32_t *elem,
                            int32_t *fill, int32_t *scan_tmp, int32_t *cell_start, int32_t *perm,
                            int2 *tmp)
{
    const int64_t ntiles = cell_tiles(E);
    if (ntiles > INT32_MAX) return set_error(FSI_ERR_ARG, "cell table: too many cells");
    int32_t *tile_sum = scan_tmp + kScanHdr;
    tile_sums_kernel<<<(int)ntiles, kLbThreads, 0, s>>>(E, fill, tile_sum);
    FSI_TRY(check_launch("cell tile sums kernel"));
    if (ntiles <= kDirectTiles) {
        tile_scan_kernel<true><<<(int)ntiles, kLbThreads, 0, s>>>(E, fill, tile_sum, cell_start);
    } else {
        tile_prefix_kernel<<<1, 1024, 0, s>>>(ntiles, tile_sum);
        FSI_TRY(check_launch("cell tile prefix kernel"));
        tile_scan_kernel<false><<<(int)ntiles, kLbThreads, 0, s>>>(E, fill, tile_sum, cell_start);
    }
    FSI_TRY(check_launch("cell scan kernel"));
    if (m > 0 && tmp) {
        scatter_arrival_kernel<<<blocks_for(m, 256), 256, 0, s>>>(m, E, elem, perm, cell_start,
                                                                  fill, scan_tmp, tmp);
        FSI_TRY(check_launch("scatter kernel"));
        rank_place_kernel<<<blocks_for(m, 256, sm_count() * 32), 256, 0, s>>>(
            m, E, cell_start, tmp, perm, fill, scan_tmp);
        FSI_TRY(check_launch("rank place kernel"));
        if (m > kWarpSortMax) {
            const int smem = kBlockSortMax * (int)sizeof(int32_t);
            FSI_TRY(set_smem_limit((const void *)dense_pairs_kernel, smem));
            dense_pairs_kernel<<<sm_count(), 1024, smem, s>>>(E, m, cell_start, tmp, perm, fill,
                                                             scan_tmp);
            FSI_TRY(check_launch("dense cell sort kernel"));
        }
    } else if (m > 0) {
        scatter_down_kernel<<<blocks_for(m, 256), 256, 0, s>>>(m, E, elem, cell_start, fill,
                                                               scan_tmp, perm);
        FSI_TRY(check_launch("scatter kernel"));
        // the counters are back to zero: their head lists the cells too full
        // for a warp, scan_tmp[0] counts them
        cell_sort_kernel<<<blocks_for((E + 32) / 32 * 32, kSortThreads, sm_count() * 16),
                           kSortThreads, 0, s>>>(E, m, cell_start, perm, fill, scan_tmp);
        FSI_TRY(check_launch("cell sort kernel"));
        if (m > kWarpSortMax) {
            const int smem = kBlockSortMax * (int)sizeof(int32_t);
            FSI_TRY(set_smem_limit((const void *)dense_sort_kernel, smem));
            dense_sort_kernel<<<sm_count(), 1024, smem, s>>>(E, m, cell_start, perm, fill,
                                                            scan_tmp);
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
    const bool table = cell_start != nullptr;
    // with a table the outside points are its tail [cell_start[E], m): no
    // separate counter (and no clearing launch) is needed
    unsigned long long *nout = nullptr;
    if (!table && (n_outside || strict)) {
        nout = (unsigned long long *)mesh->dev_counters;
        FSI_CUDA(cudaMemsetAsync(nout, 0, sizeof(unsigned long long), s), "memset");
    }
    if (table && !mesh->hash_clean)
        FSI_CUDA(cudaMemsetAsync(mesh->hash_fill, 0, (E + 1) * sizeof(int32_t), s), "memset");
    if (table) mesh->hash_clean = false;
    if (table && m > mesh->pt_tmp_cap) {
        // grow-only point scratch of the cell table: (point, cell) pairs
        cudaFree(mesh->pt_tmp);
        mesh->pt_tmp = nullptr;
        mesh->pt_tmp_cap = 0;
        const int64_t cap = std::max<int64_t>(m, 1024);
        FSI_CUDA(cudaMalloc(&mesh->pt_tmp, cap * sizeof(int2)), "point scratch");
        mesh->pt_tmp_cap = cap;
    }
    GridArgs g = grid_args(mesh);
    if (m > 0 && mesh->coords64) {
        locate_mapped_kernel<<<blocks_for(m, 128), 128, 0, s>>>(
            m, g, (const double4 *)mesh->coords64, X, elem, xi,
            table ? mesh->hash_fill : nullptr, nout, table ? perm : nullptr);
        FSI_TRY(check_launch("locate kernel"));
    } else if (m > 0) {
        FSI_TRY(launch_locate(s, m, g, X, elem, xi, table ? mesh->hash_fill : nullptr, nout,
                              table ? perm : nullptr));
    }
    if (table) {
        FSI_TRY(build_cell_table(s, E, m, elem, mesh->hash_fill, mesh->scan_tmp, cell_start, perm,
                                 mesh->pt_tmp));
        mesh->hash_clean = true;
    }
    if (n_outside || strict) {
        unsigned long long h = 0;
        if (table) {
            int32_t inside = 0;
            FSI_CUDA(cudaMemcpyAsync(&inside, cell_start + E, sizeof inside,
                                     cudaMemcpyDeviceToHost, s), "memcpy");
            FSI_CUDA(cudaStreamSynchronize(s), "stream sync");
            h = (unsigned long long)(m - inside);
        } else {
            FSI_CUDA(cudaMemcpyAsync(&h, nout, sizeof h, cudaMemcpyDeviceToHost, s), "memcpy");
            FSI_CUDA(cudaStreamSynchronize(s), "stream sync");
        }
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
        FSI_TRY(launch_locate(s, m, g, X, elem, xi, table ? fill : nullptr, nout));
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
