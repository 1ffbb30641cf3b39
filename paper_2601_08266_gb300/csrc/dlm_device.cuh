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
            ux += Na * to_c<T>(v.x);
            uy += Na * to_c<T>(v.y);
            uz += Na * to_c<T>(v.z);
        }
    }
    u[3 * b] = to_s(ux);
    u[3 * b + 1] = to_s(uy);
    u[3 * b + 2] = to_s(uz);
}

// Spreading, pass 1: one warp per segment of 32 consecutive cells.  For each
// occupied cell the lanes stride over its points (perm order) and accumulate the
// 8 corner contributions w_B N_a(xi_B) lambda_B (24 values), then a butterfly
// reduction (fixed lane order, so deterministic) gives the cell's corner sums
// S[cell][8][3].
// (called by all 32 lanes of a warp for the segment of cells [c0, c0+32))
// T is the compute type; inputs are in StorageOf<T> (FP64 for double-float).
template <typename T>
__device__ __forceinline__ void spread_cells_segment(
    int64_t E, int64_t c0, const typename StorageOf<T>::type *__restrict__ xi,
    const int32_t *__restrict__ start, const int32_t *__restrict__ perm,
    const typename StorageOf<T>::type *__restrict__ lam,
    const typename StorageOf<T>::type *__restrict__ w, T *__restrict__ S)
{
    const int lane = threadIdx.x & 31;
    {
        const int64_t myc = c0 + lane;
        int lo = 0, hi = 0;
        if (myc < E) {
            lo = start[myc];
            hi = start[myc + 1];
        }
        unsigned occ = __ballot_sync(0xffffffffu, hi > lo);
        while (occ) {
            const int l = __ffs(occ) - 1;
            occ &= occ - 1;
            const int plo = __shfl_sync(0xffffffffu, lo, l);
            const int phi = __shfl_sync(0xffffffffu, hi, l);
            T acc[24];
#pragma unroll
            for (int k = 0; k < 24; ++k) acc[k] = T(0);
            for (int p = plo + lane; p < phi; p += 32) {
                const int b = perm[p];
                const T x0 = to_c<T>(xi[3 * b]), x1 = to_c<T>(xi[3 * b + 1]),
                        x2 = to_c<T>(xi[3 * b + 2]);
                const T s = w ? to_c<T>(w[b]) * T(0.125f) : T(0.125f);
                const T l0 = to_c<T>(lam[3 * b]), l1 = to_c<T>(lam[3 * b + 1]),
                        l2 = to_c<T>(lam[3 * b + 2]);
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const T Na = shape_1d(x0, a & 1) * shape_1d(x1, (a >> 1) & 1) *
                                 shape_1d(x2, (a >> 2) & 1) * s;
                    acc[3 * a] += Na * l0;
                    acc[3 * a + 1] += Na * l1;
                    acc[3 * a + 2] += Na * l2;
                }
            }
            // transpose-reduce across the warp: each level halves the values a
            // lane carries (12, 6, 3), then a butterfly over the last two bits;
            // the pattern is fixed, so the sums are deterministic.
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
                T *dst = S + (c0 + l) * 24 + idx0;
                dst[0] = acc[0];
                dst[1] = acc[1];
                dst[2] = acc[2];
            }
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
