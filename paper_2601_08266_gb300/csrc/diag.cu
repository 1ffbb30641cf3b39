// diag.cu -- the nodal diagonal blocks of the VMS Jacobian (Sec. 2.4, the
// linearised weak form) on the uniform grid, computed directly instead of by
// probing.
//
// The block of node a is J_aa[r][c] = dR_(a,r) / dy_(a,c): the response of
// node a's own rows to the unit direction e_c at node a.  Probing gets it from
// 8 colours x 3 (or 4) full Jacobian applies.  Here one pass per element
// colour forms it from its definition: at every Gauss point the base state
// (tau_M, tau_C, fine scales) once, then for each of the element's 8 nodes a
// and each column c the linearised Gauss-point terms of the unit direction
// (dv = c_v N_a e_c, grad dv = c_v e_c (x) grad N_a, da = c_a N_a e_c; for
// the pressure column dp = N_a, grad dp = grad N_a), projected on node a's
// own test function only.  The terms are those of the Jacobian apply with the
// direction's zeros taken out (about 80 operations instead of 110), and no
// evaluation or projection butterflies are needed, so a block column costs
// about a tenth of a Jacobian apply.
//
// Layout: eight lanes per element (lane g = node g, then Gauss point g), the
// lanes' contributions to a node summed by a three-level butterfly, node by
// node, so that lane a ends with node a's columns.  Elements of one parity colour
// share no node, so each colour pass adds its elements' blocks to the node
// blocks without conflicts; the eight passes run in a fixed order, and the
// result is deterministic (no atomics).
#include <type_traits>

#include "fsi_internal.cuh"

#include "vms_device.cuh"

namespace fsi {
namespace {

using namespace vmsd;

// Per-Gauss-point constants of the linearisation that do not depend on the
// direction: d tau_M = K1 v.G dv, d tau_C = K2 d tau_M, and the convective
// weight mw_j = -rho (v_j + u'_j).
template <typename T> struct DiagGP {
    T K1, K2, mw[3];
};

// Linearised Gauss-point terms X (value coefficients) and Y (gradient
// coefficients) of the 4 residual rows for the unit direction of column C of
// a node whose shape value and gradient here are N and dN: the
// directional derivative of gp_residual_terms (the same expressions as
// gp_jacobian_terms) with the direction's zero entries dropped.
template <typename T, int C>
__device__ __forceinline__ void unit_terms(const VmsArgs<T> &P, const GP<T> &q,
                                           const DiagGP<T> &k, T N, const T (&dN)[3],
                                           T (&X)[4], T (&Y)[4][3])
{
    if constexpr (C < 3) {
        // velocity column: dv = n e_C, d grad v = e_C (x) dn, da = an e_C
        const T n = P.c_v * N, an = P.c_a * N;
        const T dn[3] = {P.c_v * dN[0], P.c_v * dN[1], P.c_v * dN[2]};
        // dv.grad v_i + v.grad dv_i + da_i
        T dadc[3];
        for (int i = 0; i < 3; ++i) dadc[i] = n * q.gv[i][C];
        dadc[C] = dadc[C] + (an + dot3_t(q.v[0], dn[0], q.v[1], dn[1], q.v[2], dn[2]));
        const T GC = C == 0 ? P.G0 : (C == 1 ? P.G1 : P.G2);
        const T dtauM = k.K1 * (GC * q.v[C] * n);
        const T dtauC = k.K2 * dtauM;
        const T ka = -dtauM * P.inv_rho;
        T dup[3];
        for (int i = 0; i < 3; ++i) dup[i] = fma_t(ka, q.rM[i], q.cup * (P.rho * dadc[i]));
        const T drC = dn[C];
        const T dpp = -P.rho * dot2_t(dtauC, q.rC, q.tauC, drC);
        for (int i = 0; i < 3; ++i) {
            T t = dadc[i];
            t = fma_t(dup[0], q.gv[i][0], t);
            t = fma_t(dup[1], q.gv[i][1], t);
            t = fma_t(dup[2], q.gv[i][2], t);
            if (i == C) t = t + dot3_t(q.up[0], dn[0], q.up[1], dn[1], q.up[2], dn[2]);
            X[i] = P.rho * t;
        }
        X[3] = drC;
        T md[3];
        for (int j = 0; j < 3; ++j) md[j] = -P.rho * dup[j];
        md[C] = md[C] - P.rho * n;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                T t = fma_t(md[j], q.up[i], k.mw[j] * dup[i]);
                if (i == C) t = fma_t(P.mu, dn[j], t);
                if (j == C) t = fma_t(P.mu, dn[i], t);
                Y[i][j] = t;
            }
        for (int i = 0; i < 3; ++i) Y[i][i] = Y[i][i] - dpp;
        for (int j = 0; j < 3; ++j) Y[3][j] = -dup[j];
    } else {
        // pressure column: dp = N, grad dp = dN (d tau = 0, dp' = 0)
        T dup[3];
        for (int i = 0; i < 3; ++i) dup[i] = q.cup * dN[i];
        for (int i = 0; i < 3; ++i)
            X[i] = P.rho * dot3_t(dup[0], q.gv[i][0], dup[1], q.gv[i][1], dup[2], q.gv[i][2]);
        X[3] = T(0);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Y[i][j] = fma_t(-P.rho * dup[j], q.up[i], k.mw[j] * dup[i]);
        for (int i = 0; i < 3; ++i) Y[i][i] = Y[i][i] - N;
        for (int j = 0; j < 3; ++j) Y[3][j] = -dup[j];
    }
}

// Column C of the element's contribution to the diagonal block of this lane's
// node, rows 0..R-1: for each of the 8 nodes a in turn, every lane (Gauss
// point g) forms its point's contribution (unit direction of node a,
// projected on node a's test function), a butterfly over the lane bits
// (4, 2, 1) sums the 8 points (the same value in every lane: each level adds
// the same two partial sums), and lane a keeps it.  One node at a time keeps
// the registers to one column's rows (the 8-node transposed reduction held
// 8 x R values and took all 255 registers).
template <typename T, int C, int R>
__device__ __forceinline__ void diag_column(const VmsArgs<T> &P, const GP<T> &q,
                                            const DiagGP<T> &k, int g, T (&out)[R])
{
    const int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = T(0);
#pragma unroll 1
    for (int a = 0; a < 8; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        // 1D factors at this Gauss point: kB1 on the node's side, kB2 across
        const T bx = ax == gx ? cB1<T>() : cB2<T>();
        const T by = ay == gy ? cB1<T>() : cB2<T>();
        const T bz = az == gz ? cB1<T>() : cB2<T>();
        const T N = bx * by * bz;
        const T dN[3] = {(ax ? P.ih0 : -P.ih0) * (by * bz), (ay ? P.ih1 : -P.ih1) * (bx * bz),
                         (az ? P.ih2 : -P.ih2) * (bx * by)};
        T X[4], Y[4][3];
        unit_terms<T, C>(P, q, k, N, dN, X, Y);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T t = fma_t(Y[r][2], dN[2], fma_t(Y[r][1], dN[1], fma_t(Y[r][0], dN[0], X[r] * N)));
            t = t + shx(t, 4);
            t = t + shx(t, 2);
            t = t + shx(t, 1);
            if (a == g) out[r] = P.detJ * t;
        }
    }
}

// One colour pass: elements (ex, ey, ez) with ex = ox (mod 2), ... (colour =
// ox + 2 oy + 4 oz) add their contributions to blocks [n][4][4] (row-major,
// columns 0..NC-1, rows 0..NC-1).  The loop bound is uniform over the block,
// so every lane reaches every shuffle.
template <typename T, int NC>
__global__ void __launch_bounds__(256) diag_blocks_kernel(const VmsArgs<T> P, int color,
                                                          T *__restrict__ blocks)
{
    constexpr bool OUT = false;
    const int g = threadIdx.x & 7;
    const int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
    const T sx = gx ? P.ih0 : -P.ih0, sy = gy ? P.ih1 : -P.ih1, sz = gz ? P.ih2 : -P.ih2;
    const int ox = color & 1, oy = (color >> 1) & 1, oz = (color >> 2) & 1;
    const int64_t cx = (P.Nx - ox + 1) / 2, cy = (P.Ny - oy + 1) / 2, cz = (P.Nz - oz + 1) / 2;
    const int64_t EC = cx * cy * cz;
    const int64_t NX1 = P.Nx + 1, NXY1 = NX1 * (P.Ny + 1);
    const int64_t per_block = blockDim.x >> 3, stride = (int64_t)gridDim.x * per_block;
    for (int64_t base = blockIdx.x * per_block; base < EC; base += stride) {
        const int64_t e = base + (threadIdx.x >> 3);
        const bool valid = e < EC;
        const int64_t ex = ox + 2 * (valid ? e % cx : 0);
        const int64_t ey = oy + 2 * (valid ? (e / cx) % cy : 0);
        const int64_t ez = oz + 2 * (valid ? e / (cx * cy) : 0);
        const int64_t node = (ex + gx) + NX1 * (ey + gy) + NXY1 * (ez + gz);
        const vec4<T> zero = {T(0), T(0), T(0), T(0)};
        const vec4<T> u = valid ? load_c<T>(P.U + node) : zero;
        const vec4<T> ac = valid ? load_c<T>(P.A + node) : zero;
        const vec4<T> ff = (valid && P.f) ? load_c<T>(P.f + node) : zero;
        // the Gauss-point state of the Jacobian apply (brick_body's evaluation)
        GP<T> q;
        {
            VG<T> e0, e1, e2, e3;
            eval_vg4<OUT>(u, sx, sy, sz, e0, e1, e2, e3);
            q.v[0] = e0.v; q.gv[0][0] = e0.gx; q.gv[0][1] = e0.gy; q.gv[0][2] = e0.gz;
            q.v[1] = e1.v; q.gv[1][0] = e1.gx; q.gv[1][1] = e1.gy; q.gv[1][2] = e1.gz;
            q.v[2] = e2.v; q.gv[2][0] = e2.gx; q.gv[2][1] = e2.gy; q.gv[2][2] = e2.gz;
            q.p = e3.v; q.gp[0] = e3.gx; q.gp[1] = e3.gy; q.gp[2] = e3.gz;
        }
        eval_v2<OUT>(ac.x, ac.y, q.a[0], q.a[1]);
        q.a[2] = eval_v<OUT>(ac.z);
        q.s = P.has_s ? eval_v<OUT>(ac.w) : T(1);
        if (P.f) {
            eval_v2<OUT>(ff.x, ff.y, q.f[0], q.f[1]);
            q.f[2] = eval_v<OUT>(ff.z);
            for (int i = 0; i < 3; ++i) q.a[i] = q.a[i] - q.f[i];
        } else {
            q.f[0] = q.f[1] = q.f[2] = T(0);
        }
        if (!valid) q.s = T(1);  // keep tau finite on idle lanes
        base_state(P, q);
        DiagGP<T> k;
        k.K1 = -(q.tauM * q.tauM * q.tauM * q.s);
        k.K2 = -q.tauC * (q.s * (P.q0 + q.vGv) * q.tauM);
        for (int j = 0; j < 3; ++j) k.mw[j] = -P.rho * (q.v[j] + q.up[j]);

        T c0[NC], c1[NC], c2[NC], c3[NC];
        diag_column<T, 0, NC>(P, q, k, g, c0);
        diag_column<T, 1, NC>(P, q, k, g, c1);
        diag_column<T, 2, NC>(P, q, k, g, c2);
        if constexpr (NC == 4) diag_column<T, 3, NC>(P, q, k, g, c3);
        if (valid) {
            T *b = blocks + 16 * node;
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                b[4 * r + 0] += c0[r];
                b[4 * r + 1] += c1[r];
                b[4 * r + 2] += c2[r];
                if constexpr (NC == 4) b[4 * r + 3] += c3[r];
            }
        }
    }
}

template <typename T>
fsi_status diag_blocks_t(fsi_mesh *m, int ncols, const void *U, const void *A, const void *f,
                         T *blocks)
{
    // the brick schedule is irrelevant here (no bricks); make_args needs one
    const Brick &b = m->brick[1][std::is_same<T, double>::value ? FSI_F64 : FSI_F32];
    const VmsArgs<T> P = make_args<T>(m, b, U, A, f, nullptr, nullptr);
    cudaStream_t s = m->stream;
    FSI_CUDA(cudaMemsetAsync(blocks, 0, (size_t)m->n_nodes * 16 * sizeof(T), s), "memset");
    const int64_t per_colour = (m->n_elems + 7) / 8;
    int64_t grid = (per_colour + 31) / 32;
    if (grid > (int64_t)sm_count() * 8) grid = (int64_t)sm_count() * 8;
    if (grid < 1) grid = 1;
    for (int color = 0; color < 8; ++color) {
        if (ncols == 4)
            diag_blocks_kernel<T, 4><<<(int)grid, 256, 0, s>>>(P, color, blocks);
        else
            diag_blocks_kernel<T, 3><<<(int)grid, 256, 0, s>>>(P, color, blocks);
        FSI_TRY(check_launch("diagonal blocks kernel"));
    }
    return FSI_OK;
}

}  // namespace

fsi_status vms_diag_blocks(fsi_mesh *m, fsi_prec prec, int ncols, const void *U, const void *A,
                           const void *f, void *blocks)
{
    if (m->tet || m->coords64) return set_error(FSI_ERR_ARG, "vms_diag_blocks: uniform grid only");
    if (ncols != 3 && ncols != 4) return set_error(FSI_ERR_ARG, "vms_diag_blocks: 3 or 4 columns");
    if (prec == FSI_F64) return diag_blocks_t<double>(m, ncols, U, A, f, (double *)blocks);
    if (prec == FSI_F32) return diag_blocks_t<float>(m, ncols, U, A, f, (float *)blocks);
    return set_error(FSI_ERR_ARG, "vms_diag_blocks: FSI_F64 or FSI_F32");
}

}  // namespace fsi
