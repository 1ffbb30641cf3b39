// dlm_device.cuh -- per-work-item device code of the coupling operators,
// shared by the single-mesh kernels (dlm.cu) and the batched persistent
// kernels (batch.cu).  See dlm.cu for the design.
#pragma once

#include "df64.cuh"
#include "fsi_internal.cuh"

namespace fsi {
namespace dlmd {

struct GridArgs {
    int Nx, Ny, Nz;
    double x0, y0, z0, hx, hy, hz;
};

template <typename T> __device__ __forceinline__ T shape_1d(T xi, int side)
{
    return side ? (T(1) + xi) : (T(1) - xi);
}

// Interpolation for one point b (u = C^T V, Eq. nodal_solid_velo).  T is the
// compute type; xi, U and u are in StorageOf<T>.
template <typename T>
__device__ __forceinline__ void interp_point(
    const GridArgs &g, int64_t b, const int32_t *__restrict__ elem,
    const typename StorageOf<T>::type *__restrict__ xi,
    const vec4<typename StorageOf<T>::type> *__restrict__ U,
    typename StorageOf<T>::type *__restrict__ u)
{
    const int NX1 = g.Nx + 1, NXY1 = (g.Nx + 1) * (g.Ny + 1);
    const int E = g.Nx * g.Ny * g.Nz;
    const int e = elem[b];
    T ux = T(0), uy = T(0), uz = T(0);
    if (e >= 0 && e < E) {
        const int ex = e % g.Nx, ey = (e / g.Nx) % g.Ny, ez = e / (g.Nx * g.Ny);
        const T x0 = to_c<T>(xi[3 * b]), x1 = to_c<T>(xi[3 * b + 1]),
                x2 = to_c<T>(xi[3 * b + 2]);
        const int n0 = ex + NX1 * ey + NXY1 * ez;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
            const T Na = shape_1d(x0, ax) * shape_1d(x1, ay) * shape_1d(x2, az) * T(0.125f);
            const auto v = ld4(U + n0 + ax + NX1 * ay + NXY1 * az);
            ux = madd(Na, to_c<T>(v.x), ux);
            uy = madd(Na, to_c<T>(v.y), uy);
            uz = madd(Na, to_c<T>(v.z), uz);
        }
    }
    u[3 * b] = to_s(ux);
    u[3 * b + 1] = to_s(uy);
    u[3 * b + 2] = to_s(uz);
}

// Corner contributions w_B N_a(xi_B) lambda_B of one point B added to acc
// (T the compute type; inputs in StorageOf<T>).
template <typename T>
__device__ __forceinline__ void spread_accumulate(
    int b, const typename StorageOf<T>::type *__restrict__ xi,
    const typename StorageOf<T>::type *__restrict__ lam,
    const typename StorageOf<T>::type *__restrict__ w, T (&acc)[24])
{
    const T x0 = to_c<T>(xi[3 * b]), x1 = to_c<T>(xi[3 * b + 1]), x2 = to_c<T>(xi[3 * b + 2]);
    const T s = w ? to_c<T>(w[b]) * T(0.125f) : T(0.125f);
    const T l0 = to_c<T>(lam[3 * b]), l1 = to_c<T>(lam[3 * b + 1]), l2 = to_c<T>(lam[3 * b + 2]);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const T Na = shape_1d(x0, a & 1) * shape_1d(x1, (a >> 1) & 1) *
                     shape_1d(x2, (a >> 2) & 1) * s;
        acc[3 * a] = madd(Na, l0, acc[3 * a]);
        acc[3 * a + 1] = madd(Na, l1, acc[3 * a + 1]);
        acc[3 * a + 2] = madd(Na, l2, acc[3 * a + 2]);
    }
}

// Spreading, pass 1, on one segment of kSpreadSeg = 8 consecutive cells
// (called by all 32 lanes of a warp for the cells [c0, c0 + 8)).  Four lanes
// share a cell of at most kGroupCell points: lane k of the group sums the
// cell's points k, k+4, ... (perm order) into the 8 corner contributions
// w_B N_a(xi_B) lambda_B (24 values), then a two-level transpose-reduce over
// the group leaves 6 corner sums in each lane.  Fuller cells are taken by the
// whole warp: the lanes stride over the points and a five-level
// transpose-reduce gives the sums.  Every cell's corner sums S[cell][8][3]
// come out of a fixed order of operations, so the result is deterministic.
// (Thin leaflets occupy few cells of few rows: short segments spread them
// over more warps.)
constexpr int kSpreadSeg = 8;
constexpr int kGroupCell = 128;

template <typename T>
__device__ __forceinline__ void spread_cells_segment(
    int64_t E, int64_t c0, const typename StorageOf<T>::type *__restrict__ xi,
    const int32_t *__restrict__ start, const int32_t *__restrict__ perm,
    const typename StorageOf<T>::type *__restrict__ lam,
    const typename StorageOf<T>::type *__restrict__ w, T *__restrict__ S)
{
    const int lane = threadIdx.x & 31;
    const int64_t myc = c0 + (lane >> 2);
    int lo = 0, hi = 0;
    if (myc < E) {
        lo = start[myc];
        hi = start[myc + 1];
    }
    if (__all_sync(0xffffffffu, hi == lo)) return;
    {
        const bool group = hi - lo <= kGroupCell;
        T acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = T(0);
        if (group)
            for (int p = lo + (lane & 3); p < hi; p += 4) spread_accumulate<T>(perm[p], xi, lam, w, acc);
        const bool b1 = lane & 2, b0 = lane & 1;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const T send = b1 ? acc[k] : acc[12 + k];
            const T keep = b1 ? acc[12 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 2);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T send = b0 ? acc[k] : acc[6 + k];
            const T keep = b0 ? acc[6 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 1);
        }
        if (group && hi > lo) {
            T *dst = S + myc * 24 + (b1 ? 12 : 0) + (b0 ? 6 : 0);
#pragma unroll
            for (int k = 0; k < 6; ++k) dst[k] = acc[k];
        }
    }
    // fuller cells: the whole warp, one cell after the other
    unsigned occ = __ballot_sync(0xffffffffu, hi - lo > kGroupCell && (lane & 3) == 0);
    while (occ) {
        const int l = __ffs(occ) - 1;
        occ &= occ - 1;
        const int plo = __shfl_sync(0xffffffffu, lo, l);
        const int phi = __shfl_sync(0xffffffffu, hi, l);
        T acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = T(0);
        for (int p = plo + lane; p < phi; p += 32) spread_accumulate<T>(perm[p], xi, lam, w, acc);
        // each level halves the values a lane carries (12, 6, 3), then a
        // butterfly over the last two bits
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const T send = b4 ? acc[k] : acc[12 + k];
            const T keep = b4 ? acc[12 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 16);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T send = b3 ? acc[k] : acc[6 + k];
            const T keep = b3 ? acc[6 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 8);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T send = b2 ? acc[k] : acc[3 + k];
            const T keep = b2 ? acc[3 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 4);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[k] = acc[k] + shfl_x(acc[k], 2);
            acc[k] = acc[k] + shfl_x(acc[k], 1);
        }
        if ((lane & 3) == 0) {
            const int idx0 = (b4 ? 12 : 0) + (b3 ? 6 : 0) + (b2 ? 3 : 0);
            T *dst = S + (c0 + (l >> 2)) * 24 + idx0;
            dst[0] = acc[0];
            dst[1] = acc[1];
            dst[2] = acc[2];
        }
    }
}

// Spreading, pass 2: every node sums the corner sums of its (up to 8)
// occupied cells in a fixed order.
template <typename T>
__device__ __forceinline__ void spread_node(const GridArgs &g, int node,
                                            const int32_t *__restrict__ start,
                                            const T *__restrict__ S,
                                            typename StorageOf<T>::type *__restrict__ F,
                                            int accumulate)
{
    const int NX1 = g.Nx + 1, NY1 = g.Ny + 1;
    {
        const int i = node % NX1, j = (node / NX1) % NY1, k = node / (NX1 * NY1);
        T fx = T(0), fy = T(0), fz = T(0);
        bool touched = false;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            // this node is local corner (cx,cy,cz) of cell (i-cx, j-cy, k-cz)
            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
            const int ex = i - cx, ey = j - cy, ez = k - cz;
            if (ex < 0 || ey < 0 || ez < 0 || ex >= g.Nx || ey >= g.Ny || ez >= g.Nz) continue;
            const int cell = ex + g.Nx * (ey + g.Ny * ez);
            if (start[cell + 1] == start[cell]) continue;
            const T *sc = S + (size_t)cell * 24 + 3 * c;
            fx = fx + sc[0];
            fy = fy + sc[1];
            fz = fz + sc[2];
            touched = true;
        }
        auto *o = F + 4 * (size_t)node;
        if (accumulate) {
            if (touched) {
                o[0] = to_s(to_c<T>(o[0]) + fx);
                o[1] = to_s(to_c<T>(o[1]) + fy);
                o[2] = to_s(to_c<T>(o[2]) + fz);
            }
        } else {
            o[0] = to_s(fx);
            o[1] = to_s(fy);
            o[2] = to_s(fz);
        }
    }
}

}  // namespace dlmd
}  // namespace fsi
