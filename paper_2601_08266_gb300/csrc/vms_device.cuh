// vms_device.cuh -- per-work-item device code of the VMS operators, shared by
// the single-mesh kernels (vms.cu) and the batched persistent kernels
// (batch.cu).  See vms.cu for the design.
#pragma once

#include <type_traits>

#include "df64.cuh"
#include "fsi_internal.cuh"
#include "pairs.cuh"

namespace fsi {
namespace vmsd {

constexpr double kQ = 0.57735026918962576451;  // 1/sqrt(3): Gauss abscissa
constexpr double kB1 = 0.5 * (1.0 + kQ);      // 1D linear basis at the near point
constexpr double kB2 = 0.5 * (1.0 - kQ);      // ... at the far point
// the same constants as exact float pairs (split at compile time)
constexpr float kB1h = static_cast<float>(kB1);
constexpr float kB1l = static_cast<float>(kB1 - static_cast<double>(kB1h));
constexpr float kB2h = static_cast<float>(kB2);
constexpr float kB2l = static_cast<float>(kB2 - static_cast<double>(kB2h));

template <typename T> __device__ __forceinline__ T cB1() { return T(kB1); }
template <typename T> __device__ __forceinline__ T cB2() { return T(kB2); }
template <> __device__ __forceinline__ df64 cB1<df64>() { return df64(kB1h, kB1l); }
template <> __device__ __forceinline__ df64 cB2<df64>() { return df64(kB2h, kB2l); }

// node record of double-float values (two float4 loads)
__device__ __forceinline__ vec4<df64> ld4_df(const vec4<df64> *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    return {df64(a.x, a.y), df64(a.z, a.w), df64(b.x, b.y), df64(b.z, b.w)};
}
template <typename T> __device__ __forceinline__ vec4<T> ld4_blk(const vec4<T> *p) { return ld4(p); }
template <> __device__ __forceinline__ vec4<df64> ld4_blk<df64>(const vec4<df64> *p)
{
    return ld4_df(p);
}

// Per-Gauss-point geometry of a mapped grid, built once per coordinate set and
// compute type and read by the VMS kernels: Ji[9] (row-major), G00 G01 G02 G11
// G12 G22, G:G, 1/tr G, det J.  Layout [element][value][Gauss point], so the 8
// lanes of an element read 8 consecutive entries per value.  Double-float
// entries are stored as (hi, lo) float pairs.
constexpr int kMapGeo = 18;
template <typename T> struct GeoStore {
    using type = T;
};
template <> struct GeoStore<df64> {
    using type = float2;
};
template <typename T> __device__ __forceinline__ T geo_ld(const typename GeoStore<T>::type *p)
{
    return __ldg(p);
}
template <> __device__ __forceinline__ df64 geo_ld<df64>(const float2 *p)
{
    const float2 v = __ldg(p);
    return df64(v.x, v.y);
}
template <typename T> __device__ __forceinline__ typename GeoStore<T>::type geo_st(T v) { return v; }
template <> __device__ __forceinline__ float2 geo_st<df64>(df64 v) { return make_float2(v.hi, v.lo); }

template <typename T> struct VmsArgs {
    using S = typename StorageOf<T>::type;
    int Nx, Ny, Nz;
    int bx, by, bz;
    int nbx, nby, nbz;
    T rho, mu, inv_rho;
    T G0, G1, G2, inv_trG, q0;  // q0 = C_T/dt^2 + C_I (mu/rho)^2 G:G
    T ih0, ih1, ih2;            // 1/h_k
    T detJ;
    T c_a, c_v;                 // d A / d y_v, d U / d y_v
    T c_av;                     // c_a / c_v
    T ct_dt2, CInu2;            // C_T/dt^2 and C_I (mu/rho)^2 (mapped grids: G per Gauss point)
    int has_s;
    const vec4<S> *Xc;          // mapped grids: node coordinates [n][4] (x, y, z, 0), else null
    const typename GeoStore<T>::type *geo;  // mapped grids: [E][kMapGeo][8] Gauss-point geometry
    const vec4<S> *U, *A, *f, *x;
    vec4<T> *blocks;  // [n_bricks][(bx+1)(by+1)(bz+1)], in the compute type
    vec4<S> *out;     // [n]
    // fused residual + Jacobian apply: the residual's node blocks and output
    vec4<T> *blocks2;
    vec4<S> *out2;
};

// a b + c and a b + c d: plain expressions (contracted to FMAs) for float and
// double, one renormalisation for double-float.
template <typename T> __device__ __forceinline__ T fma_t(T a, T b, T c) { return a * b + c; }
template <> __device__ __forceinline__ df64 fma_t<df64>(df64 a, df64 b, df64 c)
{
    return df_fma(a, b, c);
}
template <typename T> __device__ __forceinline__ T dot2_t(T a, T b, T c, T d)
{
    return a * b + c * d;
}
template <> __device__ __forceinline__ df64 dot2_t<df64>(df64 a, df64 b, df64 c, df64 d)
{
    return df_dot2(a, b, c, d);
}
// a . b over three components
template <typename T> __device__ __forceinline__ T dot3_t(T a0, T b0, T a1, T b1, T a2, T b2)
{
    return fma_t(a2, b2, dot2_t(a0, b0, a1, b1));
}

template <typename T> __device__ __forceinline__ T shx(T v, int m)
{
    return __shfl_xor_sync(0xffffffffu, v, m);
}
template <> __device__ __forceinline__ df64 shx<df64>(df64 v, int m) { return df_shfl_xor(v, m); }

// the same operations on pairs of values (pairs.cuh): two fields per call
using pd = pair2<double>;
template <> __device__ __forceinline__ f32x2 fma_t<f32x2>(f32x2 a, f32x2 b, f32x2 c)
{
    return pair_fma(a, b, c);
}
template <> __device__ __forceinline__ df64x2 fma_t<df64x2>(df64x2 a, df64x2 b, df64x2 c)
{
    return pair_fma(a, b, c);
}
template <> __device__ __forceinline__ pd fma_t<pd>(pd a, pd b, pd c) { return pair_fma(a, b, c); }
template <> __device__ __forceinline__ f32x2 dot2_t<f32x2>(f32x2 a, f32x2 b, f32x2 c, f32x2 d)
{
    return pair_dot2(a, b, c, d);
}
template <>
__device__ __forceinline__ df64x2 dot2_t<df64x2>(df64x2 a, df64x2 b, df64x2 c, df64x2 d)
{
    return pair_dot2(a, b, c, d);
}
template <> __device__ __forceinline__ pd dot2_t<pd>(pd a, pd b, pd c, pd d)
{
    return pair_dot2(a, b, c, d);
}
template <> __device__ __forceinline__ f32x2 shx<f32x2>(f32x2 v, int m) { return pair_shx(v, m); }
template <> __device__ __forceinline__ df64x2 shx<df64x2>(df64x2 v, int m) { return pair_shx(v, m); }
template <> __device__ __forceinline__ pd shx<pd>(pd v, int m) { return pair_shx(v, m); }
template <> __device__ __forceinline__ f32x2 cB1<f32x2>()
{
    return {make_float2((float)kB1, (float)kB1)};
}
template <> __device__ __forceinline__ f32x2 cB2<f32x2>()
{
    return {make_float2((float)kB2, (float)kB2)};
}
template <> __device__ __forceinline__ df64x2 cB1<df64x2>()
{
    return {make_float2(kB1h, kB1h), make_float2(kB1l, kB1l)};
}
template <> __device__ __forceinline__ df64x2 cB2<df64x2>()
{
    return {make_float2(kB2h, kB2h), make_float2(kB2l, kB2l)};
}
template <> __device__ __forceinline__ pd cB1<pd>() { return {kB1, kB1}; }
template <> __device__ __forceinline__ pd cB2<pd>() { return {kB2, kB2}; }

// one node record of storage type S as compute type T
template <typename T>
__device__ __forceinline__ vec4<T> load_c(const vec4<typename StorageOf<T>::type> *p)
{
    const auto v = ld4(p);
    return {to_c<T>(v.x), to_c<T>(v.y), to_c<T>(v.z), to_c<T>(v.w)};
}

template <typename T> struct VG {
    T v, gx, gy, gz;
};

// Value and physical gradient at this lane's Gauss point of the Q1 field whose
// value at this lane's node is u.  sx = sigma_x/h_x with sigma = +1 when the
// lane's node sits at the upper side along x (and likewise sy, sz).
template <typename T> __device__ __forceinline__ VG<T> eval_vg_body(T u, T sx, T sy, T sz)
{
    const T b1 = cB1<T>(), b2 = cB2<T>();
    T uo = shx(u, 1);
    T tB = dot2_t(b1, u, b2, uo);
    T tD = u - uo;
    T tBo = shx(tB, 2), tDo = shx(tD, 2);
    T tBB = dot2_t(b1, tB, b2, tBo);
    T tBD = tB - tBo;
    T tDB = dot2_t(b1, tD, b2, tDo);
    T tBBo = shx(tBB, 4), tBDo = shx(tBD, 4), tDBo = shx(tDB, 4);
    VG<T> r;
    r.v = dot2_t(b1, tBB, b2, tBBo);
    r.gz = sz * (tBB - tBBo);
    r.gy = sy * dot2_t(b1, tBD, b2, tBDo);
    r.gx = sx * dot2_t(b1, tDB, b2, tDBo);
    return r;
}

// Native FP64 (one FP64 instruction per multiply, add or FMA alike): with
// b1 + b2 = 1, b1 u + b2 uo = uo + b1 (u - uo), so each value-type output of a
// butterfly stage is one FMA on the difference that the gradient-type output
// needs anyway: 15 FP64 instructions per field instead of 18.
template <> __device__ __forceinline__ VG<double> eval_vg_body<double>(double u, double sx,
                                                                       double sy, double sz)
{
    const double b1 = kB1;
    const double uo = shx(u, 1);
    const double tD = u - uo;
    const double tB = fma(b1, tD, uo);
    const double tBo = shx(tB, 2), tDo = shx(tD, 2);
    const double tBD = tB - tBo;
    const double tBB = fma(b1, tBD, tBo);
    const double tDB = fma(b1, tD - tDo, tDo);
    const double tBBo = shx(tBB, 4), tBDo = shx(tBD, 4), tDBo = shx(tDB, 4);
    const double dz = tBB - tBBo;
    VG<double> r;
    r.v = fma(b1, dz, tBBo);
    r.gz = sz * dz;
    r.gy = sy * fma(b1, tBD - tBDo, tBDo);
    r.gx = sx * fma(b1, tDB - tDBo, tDBo);
    return r;
}

template <typename T> __device__ __forceinline__ T eval_v_body(T u)
{
    const T b1 = cB1<T>(), b2 = cB2<T>();
    T t = dot2_t(b1, u, b2, shx(u, 1));
    t = dot2_t(b1, t, b2, shx(t, 2));
    return dot2_t(b1, t, b2, shx(t, 4));
}

// Transposed evaluation: with X the value coefficient and (Yx, Yy, Yz) the
// gradient coefficients of one residual component at this lane's Gauss point,
// returns sum_g [N_a(g) X(g) + grad N_a(g) . Y(g)] for the lane's node a.
template <typename T>
__device__ __forceinline__ T project_body(T X, T Yx, T Yy, T Yz, T sx, T sy, T sz)
{
    const T b1 = cB1<T>(), b2 = cB2<T>();
    T Xo = shx(X, 4), Yzo = shx(Yz, 4), Yxo = shx(Yx, 4), Yyo = shx(Yy, 4);
    T P1 = fma_t(sz, Yz + Yzo, dot2_t(b1, X, b2, Xo));
    T P2 = dot2_t(b1, Yx, b2, Yxo);
    T P3 = dot2_t(b1, Yy, b2, Yyo);
    T P1o = shx(P1, 2), P2o = shx(P2, 2), P3o = shx(P3, 2);
    T Q1 = fma_t(sy, P3 + P3o, dot2_t(b1, P1, b2, P1o));
    T Q2 = dot2_t(b1, P2, b2, P2o);
    T Q1o = shx(Q1, 1), Q2o = shx(Q2, 1);
    return fma_t(sx, Q2 + Q2o, dot2_t(b1, Q1, b2, Q1o));
}

// Evaluation and projection entry points.  With OUT set, double-float calls
// one out-of-line copy of each body instead of inlining it: inlined at all 8 +
// 4 + 4 call sites the double-float Jacobian body outgrows what the
// instruction cache holds for its 16 warps per SM (out of line: -6 % at 64^3,
// -12 % at 128^3); the shorter residual body is faster inlined (+3-5 %
// out of line; 6 % on mapped grids, whose geometry comes from a table).
// float and double always inline.
template <typename T> __device__ __noinline__ VG<T> eval_vg_ool(T u, T sx, T sy, T sz)
{
    return eval_vg_body(u, sx, sy, sz);
}
template <typename T> __device__ __noinline__ T eval_v_ool(T u) { return eval_v_body(u); }
template <typename T>
__device__ __noinline__ T project_ool(T X, T Yx, T Yy, T Yz, T sx, T sy, T sz)
{
    return project_body(X, Yx, Yy, Yz, sx, sy, sz);
}
// which compute types take the out-of-line copies when OUT is set
template <typename T>
constexpr bool kOutline = std::is_same<T, df64>::value || std::is_same<T, df64x2>::value;

template <bool OUT, typename T> __device__ __forceinline__ VG<T> eval_vg(T u, T sx, T sy, T sz)
{
    if constexpr (OUT && kOutline<T>)
        return eval_vg_ool(u, sx, sy, sz);
    else
        return eval_vg_body(u, sx, sy, sz);
}
template <bool OUT, typename T> __device__ __forceinline__ T eval_v(T u)
{
    if constexpr (OUT && kOutline<T>)
        return eval_v_ool(u);
    else
        return eval_v_body(u);
}
template <bool OUT, typename T>
__device__ __forceinline__ T project(T X, T Yx, T Yy, T Yz, T sx, T sy, T sz)
{
    if constexpr (OUT && kOutline<T>)
        return project_ool(X, Yx, Yy, Yz, sx, sy, sz);
    else
        return project_body(X, Yx, Yy, Yz, sx, sy, sz);
}

// Four fields of a node record evaluated as two pairs (x, y) and (z, w):
// float and double-float pairs run on the paired FP32 instructions (3-7 %
// faster VMS kernels); double has no paired form and evaluates field by field.
template <bool OUT, typename T>
__device__ __forceinline__ void eval_vg4(const vec4<T> &u, T sx, T sy, T sz, VG<T> &e0, VG<T> &e1,
                                         VG<T> &e2, VG<T> &e3)
{
    if constexpr (std::is_same<T, double>::value) {
        e0 = eval_vg<OUT>(u.x, sx, sy, sz);
        e1 = eval_vg<OUT>(u.y, sx, sy, sz);
        e2 = eval_vg<OUT>(u.z, sx, sy, sz);
        e3 = eval_vg<OUT>(u.w, sx, sy, sz);
        return;
    }
    using PO = PairOf<T>;
    const auto px = PO::pack(sx, sx), py = PO::pack(sy, sy), pz = PO::pack(sz, sz);
    const auto a = eval_vg<OUT>(PO::pack(u.x, u.y), px, py, pz);
    const auto b = eval_vg<OUT>(PO::pack(u.z, u.w), px, py, pz);
    e0 = {PO::first(a.v), PO::first(a.gx), PO::first(a.gy), PO::first(a.gz)};
    e1 = {PO::second(a.v), PO::second(a.gx), PO::second(a.gy), PO::second(a.gz)};
    e2 = {PO::first(b.v), PO::first(b.gx), PO::first(b.gy), PO::first(b.gz)};
    e3 = {PO::second(b.v), PO::second(b.gx), PO::second(b.gy), PO::second(b.gz)};
}

// values of two fields at the Gauss point
template <bool OUT, typename T> __device__ __forceinline__ void eval_v2(T u, T w, T &ru, T &rw)
{
    if constexpr (std::is_same<T, double>::value) {
        ru = eval_v<OUT>(u);
        rw = eval_v<OUT>(w);
        return;
    }
    using PO = PairOf<T>;
    const auto r = eval_v<OUT>(PO::pack(u, w));
    ru = PO::first(r);
    rw = PO::second(r);
}

// projections of two residual components
template <bool OUT, typename T>
__device__ __forceinline__ void project2(T X0, const T (&Y0)[3], T X1, const T (&Y1)[3], T sx, T sy,
                                         T sz, T &r0, T &r1)
{
    if constexpr (std::is_same<T, double>::value) {
        r0 = project<OUT>(X0, Y0[0], Y0[1], Y0[2], sx, sy, sz);
        r1 = project<OUT>(X1, Y1[0], Y1[1], Y1[2], sx, sy, sz);
        return;
    }
    using PO = PairOf<T>;
    const auto r = project<OUT>(PO::pack(X0, X1), PO::pack(Y0[0], Y1[0]), PO::pack(Y0[1], Y1[1]),
                                PO::pack(Y0[2], Y1[2]), PO::pack(sx, sx), PO::pack(sy, sy),
                                PO::pack(sz, sz));
    r0 = PO::first(r);
    r1 = PO::second(r);
}

template <typename T> __device__ __forceinline__ T inv_t(T v) { return T(1) / v; }
template <> __device__ __forceinline__ df64 inv_t<df64>(df64 v) { return df_rcp(v); }

template <typename T> __device__ __forceinline__ T rsqrt_t(T v);
template <> __device__ __forceinline__ float rsqrt_t(float v) { return 1.0f / sqrtf(v); }
// within 1 ulp (the CUDA math library's bound), far inside the operators' 1e-12
template <> __device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }
template <> __device__ __forceinline__ df64 rsqrt_t(df64 v) { return df_rsqrt(v); }

// Base state of the VMS form at one Gauss point.
// a[] holds the acceleration minus the body force (a - f): the two enter the
// residual only as that difference; cup = -tau_M / rho (u' = cup r_M)
template <typename T> struct GP {
    T v[3], gv[3][3], p, gp[3], a[3], f[3], s;
    T rM[3], rC, conv[3], tauM, tauC, up[3], pp, vGv, cup;
};

template <typename T>
__device__ __forceinline__ void base_state(const VmsArgs<T> &P, GP<T> &q)
{
    for (int i = 0; i < 3; ++i) {
        q.conv[i] = dot3_t(q.v[0], q.gv[i][0], q.v[1], q.gv[i][1], q.v[2], q.gv[i][2]);
        q.rM[i] = fma_t(P.rho, q.a[i] + q.conv[i], q.gp[i]);
    }
    q.rC = q.gv[0][0] + q.gv[1][1] + q.gv[2][2];
    q.vGv = dot3_t(P.G0 * q.v[0], q.v[0], P.G1 * q.v[1], q.v[1], P.G2 * q.v[2], q.v[2]);
    const T S = q.s * (P.q0 + q.vGv);
    q.tauM = rsqrt_t(S);
    // tau_C = 1/(tau_M tr G) and 1/tau_M = S tau_M
    q.tauC = S * q.tauM * P.inv_trG;
    q.cup = -q.tauM * P.inv_rho;
    for (int i = 0; i < 3; ++i) q.up[i] = q.cup * q.rM[i];
    q.pp = -P.rho * q.tauC * q.rC;
}

// Geometry of one Gauss point on a mapped grid: Ji = (dx/dxi)^{-1}, det,
// the metric G = Ji^T Ji of Sec. 2.1 (full), tr G and the bracket constant.
template <typename T> struct Geo {
    T Ji[3][3], det, G[3][3], inv_trG, q0;
};

// base state with a per-Gauss-point metric (mapped grids)
template <typename T>
__device__ __forceinline__ void base_state_g(const VmsArgs<T> &P, const Geo<T> &geo, GP<T> &q)
{
    for (int i = 0; i < 3; ++i) {
        q.conv[i] = dot3_t(q.v[0], q.gv[i][0], q.v[1], q.gv[i][1], q.v[2], q.gv[i][2]);
        q.rM[i] = fma_t(P.rho, q.a[i] + q.conv[i], q.gp[i]);
    }
    q.rC = q.gv[0][0] + q.gv[1][1] + q.gv[2][2];
    T vGv = T(0);
    for (int i = 0; i < 3; ++i)
        vGv += q.v[i] * (geo.G[i][0] * q.v[0] + geo.G[i][1] * q.v[1] + geo.G[i][2] * q.v[2]);
    q.vGv = vGv;
    const T S = q.s * (geo.q0 + q.vGv);
    q.tauM = rsqrt_t(S);
    q.tauC = S * q.tauM * geo.inv_trG;
    q.cup = -q.tauM * P.inv_rho;
    for (int i = 0; i < 3; ++i) q.up[i] = q.cup * q.rM[i];
    q.pp = -P.rho * q.tauC * q.rC;
}

// physical gradient from the reference one: g_j = sum_k gref_k Ji[k][j]
template <typename T>
__device__ __forceinline__ void to_phys(const Geo<T> &geo, VG<T> &e)
{
    const T a = e.gx, b = e.gy, c = e.gz;
    e.gx = a * geo.Ji[0][0] + b * geo.Ji[1][0] + c * geo.Ji[2][0];
    e.gy = a * geo.Ji[0][1] + b * geo.Ji[1][1] + c * geo.Ji[2][1];
    e.gz = a * geo.Ji[0][2] + b * geo.Ji[1][2] + c * geo.Ji[2][2];
}

// Geometry at this lane's Gauss point from the node coordinates xc of the
// element (lane = node on entry): J = dx/dxi by the butterfly (sx, sy, sz the
// reference gradient signs +-1/2), Ji by cofactors, G = Ji^T Ji, G:G, 1/tr G.
template <bool OUT, typename T>
__device__ __forceinline__ void mapped_geometry(const vec4<T> &xc, T sx, T sy, T sz,
                                                T (&out)[kMapGeo])
{
    VG<T> cx, cy, cz, cw;
    eval_vg4<OUT>(xc, sx, sy, sz, cx, cy, cz, cw);
    const T J[3][3] = {{cx.gx, cx.gy, cx.gz}, {cy.gx, cy.gy, cy.gz}, {cz.gx, cz.gy, cz.gz}};
    const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const T id = inv_t(det);
    T Ji[3][3];
    Ji[0][0] = c00 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][0] = c01 * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][0] = c02 * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    T G[3][3], GG = T(0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const T gij = Ji[0][i] * Ji[0][j] + Ji[1][i] * Ji[1][j] + Ji[2][i] * Ji[2][j];
            G[i][j] = gij;
            GG += gij * gij;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[3 * i + j] = Ji[i][j];
    out[9] = G[0][0];
    out[10] = G[0][1];
    out[11] = G[0][2];
    out[12] = G[1][1];
    out[13] = G[1][2];
    out[14] = G[2][2];
    out[15] = GG;
    out[16] = inv_t(G[0][0] + G[1][1] + G[2][2]);
    out[17] = det;
}

// Test-function coefficients of the residual at one quadrature point: X
// multiplies N_A, Y[c][j] multiplies dN_A/dx_j for residual component c.
template <typename T>
__device__ __forceinline__ void gp_residual_terms(const VmsArgs<T> &P, const GP<T> &q, T (&X)[4],
                                                  T (&Y)[4][3])
{
    // X_i = rho (a - f + v.grad v_i + u'.grad v_i), the sums in FMA order
    for (int i = 0; i < 3; ++i) {
        T t = q.a[i] + q.conv[i];
        t = fma_t(q.up[0], q.gv[i][0], t);
        t = fma_t(q.up[1], q.gv[i][1], t);
        t = fma_t(q.up[2], q.gv[i][2], t);
        X[i] = P.rho * t;
    }
    // Y_ij = mu (d_j v_i + d_i v_j) - rho (v_j + u'_j) u'_i: the symmetric
    // viscous part once per pair
    T mw[3];
    for (int j = 0; j < 3; ++j) mw[j] = -P.rho * (q.v[j] + q.up[j]);
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            const T muS = P.mu * (q.gv[i][j] + q.gv[j][i]);
            Y[i][j] = fma_t(mw[j], q.up[i], muS);
            if (j != i) Y[j][i] = fma_t(mw[i], q.up[j], muS);
        }
    for (int i = 0; i < 3; ++i) Y[i][i] -= q.p + q.pp;
    X[3] = q.rC;
    for (int j = 0; j < 3; ++j) Y[3][j] = -q.up[j];
}

// v . G dv with the full metric of a Gauss point
template <typename T>
__device__ __forceinline__ T vGdv_full(const Geo<T> &geo, const GP<T> &q, const T (&dv)[3])
{
    T vGdv = T(0);
    for (int i = 0; i < 3; ++i)
        vGdv += q.v[i] * (geo.G[i][0] * dv[0] + geo.G[i][1] * dv[1] + geo.G[i][2] * dv[2]);
    return vGdv;
}

// The same coefficients of the Jacobian in the direction (dv, grad dv, da, dp,
// grad dp) (physical gradients, chain factors applied); vGdv = v . G dv and
// q0 = C_T/dt^2 + C_I nu^2 G:G at this point.
template <typename T>
__device__ __forceinline__ void gp_jacobian_terms(const VmsArgs<T> &P, const GP<T> &q,
                                                  const T (&dv)[3], const T (&dgv)[3][3],
                                                  const T (&da)[3], T dp, const T (&dgp)[3],
                                                  T vGdv, T q0, T (&X)[4], T (&Y)[4][3])
{
    T dconv[3], drM[3], dup[3], dadc[3];
    for (int i = 0; i < 3; ++i) {
        // dv.grad v_i + v.grad dv_i, one product and five FMAs
        T t = q.v[0] * dgv[i][0];
        t = fma_t(q.v[1], dgv[i][1], t);
        t = fma_t(q.v[2], dgv[i][2], t);
        t = fma_t(dv[0], q.gv[i][0], t);
        t = fma_t(dv[1], q.gv[i][1], t);
        dconv[i] = fma_t(dv[2], q.gv[i][2], t);
        dadc[i] = da[i] + dconv[i];
        drM[i] = fma_t(P.rho, dadc[i], dgp[i]);
    }
    const T drC = dgv[0][0] + dgv[1][1] + dgv[2][2];
    const T dtauM = -q.tauM * q.tauM * q.tauM * q.s * vGdv;
    // d tau_C = -tau_C d tau_M / tau_M, 1/tau_M = s (q0 + vGv) tau_M
    const T dtauC = -q.tauC * dtauM * (q.s * (q0 + q.vGv) * q.tauM);
    // du' = -(d tau_M r_M + tau_M d r_M) / rho
    const T ka = -dtauM * P.inv_rho;
    for (int i = 0; i < 3; ++i) dup[i] = fma_t(ka, q.rM[i], q.cup * drM[i]);
    const T dpp = -P.rho * dot2_t(dtauC, q.rC, q.tauC, drC);
    for (int i = 0; i < 3; ++i) {
        T t = dadc[i];
        t = fma_t(dup[0], q.gv[i][0], t);
        t = fma_t(dup[1], q.gv[i][1], t);
        t = fma_t(dup[2], q.gv[i][2], t);
        t = fma_t(q.up[0], dgv[i][0], t);
        t = fma_t(q.up[1], dgv[i][1], t);
        t = fma_t(q.up[2], dgv[i][2], t);
        X[i] = P.rho * t;
    }
    // Y_ij = mu (d_j dv_i + d_i dv_j) - rho [(dv_j + du'_j) u'_i + (v_j + u'_j) du'_i]
    T mw[3], md[3];
    for (int j = 0; j < 3; ++j) {
        mw[j] = -P.rho * (q.v[j] + q.up[j]);
        md[j] = -P.rho * (dv[j] + dup[j]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            const T muS = P.mu * (dgv[i][j] + dgv[j][i]);
            Y[i][j] = fma_t(md[j], q.up[i], fma_t(mw[j], dup[i], muS));
            if (j != i) Y[j][i] = fma_t(md[i], q.up[j], fma_t(mw[i], dup[j], muS));
        }
    for (int i = 0; i < 3; ++i) Y[i][i] -= dp + dpp;
    X[3] = drC;
    for (int j = 0; j < 3; ++j) Y[3][j] = -dup[j];
}

// One brick of elements: element contributions into rel (shared memory,
// [bx*by*bz][8] node records), then the brick's node block into P.blocks.
// FUSED (with JAC): the residual at the same Gauss-point state is projected
// too, into rel + rel_records(bx*by*bz) and then P.blocks2; the evaluation of U and A
// and the base state are shared by the two operators.
// Element records in shared memory, corner-major with one padding record
// per corner row: corner c of brick element `slot` at c (nel + 1) + slot.
// The 8 lanes of an element then store to 8 different bank groups, and the
// node sums read consecutive elements from consecutive threads (element-major
// records, 8 apart, put a warp's 32 reads on the same banks: 8-way conflicts).
__host__ __device__ __forceinline__ int rel_records(int nel) { return 8 * (nel + 1); }
__device__ __forceinline__ int rel_at(int nel, int slot, int c) { return c * (nel + 1) + slot; }

template <typename T, bool JAC, bool MAPPED = false, bool FUSED = false>
__device__ __forceinline__ void brick_body(const VmsArgs<T> &P, int brick, vec4<T> *rel)
{
    static_assert(!FUSED || JAC, "the fused body computes the Jacobian apply too");
    constexpr bool OUT = JAC;  // out-of-line double-float evaluation
    const int g = threadIdx.x & 7;
    const int bxi = brick % P.nbx, byi = (brick / P.nbx) % P.nby, bzi = brick / (P.nbx * P.nby);
    const int ex0 = bxi * P.bx, ey0 = byi * P.by, ez0 = bzi * P.bz;
    const int nel = P.bx * P.by * P.bz;
    const int groups = blockDim.x >> 3;
    const int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
    // gradient signs of the butterfly: physical (+-1/h) on the uniform grid,
    // reference (+-1/2 per unit of xi) on a mapped grid
    const T sx = MAPPED ? (gx ? T(0.5f) : T(-0.5f)) : (gx ? P.ih0 : -P.ih0);
    const T sy = MAPPED ? (gy ? T(0.5f) : T(-0.5f)) : (gy ? P.ih1 : -P.ih1);
    const T sz = MAPPED ? (gz ? T(0.5f) : T(-0.5f)) : (gz ? P.ih2 : -P.ih2);
    const int NX1 = P.Nx + 1, NXY1 = (P.Nx + 1) * (P.Ny + 1);

    for (int base = 0; base < nel; base += groups) {
        // the double-float body is long: a barrier per pass keeps the CTA's
        // warps on the same stretch of it (instruction-cache locality; 3-5 %
        // faster on GB300, a loss for the shorter float/double bodies)
        if constexpr (std::is_same<T, df64>::value) __syncthreads();
        const int slot = base + (threadIdx.x >> 3);
        const int lx = slot % P.bx, ly = (slot / P.bx) % P.by, lz = slot / (P.bx * P.by);
        const int ex = ex0 + lx, ey = ey0 + ly, ez = ez0 + lz;
        const bool valid = slot < nel && ex < P.Nx && ey < P.Ny && ez < P.Nz;
        const int node = valid ? (ex + gx) + NX1 * (ey + gy) + NXY1 * (ez + gz) : 0;
        const vec4<T> zero = {T(0), T(0), T(0), T(0)};
        vec4<T> u = valid ? load_c<T>(P.U + node) : zero;
        vec4<T> ac = valid ? load_c<T>(P.A + node) : zero;
        vec4<T> ff = (valid && P.f) ? load_c<T>(P.f + node) : zero;

        Geo<T> geo;
        if constexpr (MAPPED) {
            // this lane's Gauss point from the geometry table; idle lanes
            // take the identity (their result is discarded)
            T gt[kMapGeo];
            if (valid) {
                const int64_t e = ex + (int64_t)P.Nx * (ey + (int64_t)P.Ny * ez);
                const typename GeoStore<T>::type *gp = P.geo + e * (kMapGeo * 8) + g;
#pragma unroll
                for (int k = 0; k < kMapGeo; ++k) gt[k] = geo_ld<T>(gp + 8 * k);
            } else {
#pragma unroll
                for (int k = 0; k < kMapGeo; ++k) gt[k] = T(0);
                gt[0] = gt[4] = gt[8] = gt[9] = gt[12] = gt[14] = gt[17] = T(1);
                gt[15] = T(3);
                gt[16] = T(1.0f / 3.0f);
            }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) geo.Ji[i][j] = gt[3 * i + j];
            geo.G[0][0] = gt[9];
            geo.G[0][1] = geo.G[1][0] = gt[10];
            geo.G[0][2] = geo.G[2][0] = gt[11];
            geo.G[1][1] = gt[12];
            geo.G[1][2] = geo.G[2][1] = gt[13];
            geo.G[2][2] = gt[14];
            geo.q0 = P.ct_dt2 + P.CInu2 * gt[15];
            geo.inv_trG = gt[16];
            geo.det = gt[17];
        }
        GP<T> q;
        {
            VG<T> e0, e1, e2, e3;
            eval_vg4<OUT>(u, sx, sy, sz, e0, e1, e2, e3);
            if constexpr (MAPPED) {
                to_phys(geo, e0);
                to_phys(geo, e1);
                to_phys(geo, e2);
                to_phys(geo, e3);
            }
            q.v[0] = e0.v; q.gv[0][0] = e0.gx; q.gv[0][1] = e0.gy; q.gv[0][2] = e0.gz;
            q.v[1] = e1.v; q.gv[1][0] = e1.gx; q.gv[1][1] = e1.gy; q.gv[1][2] = e1.gz;
            q.v[2] = e2.v; q.gv[2][0] = e2.gx; q.gv[2][1] = e2.gy; q.gv[2][2] = e2.gz;
            q.p = e3.v; q.gp[0] = e3.gx; q.gp[1] = e3.gy; q.gp[2] = e3.gz;
        }
        eval_v2<OUT>(ac.x, ac.y, q.a[0], q.a[1]);
        if constexpr (std::is_same<T, double>::value) {
            q.a[2] = eval_v<OUT>(ac.z);
            q.s = P.has_s ? eval_v<OUT>(ac.w) : T(1);
        } else {  // the pair's second half is free
            T sv;
            eval_v2<OUT>(ac.z, ac.w, q.a[2], sv);
            q.s = P.has_s ? sv : T(1);
        }
        if (P.f) {
            eval_v2<OUT>(ff.x, ff.y, q.f[0], q.f[1]);
            q.f[2] = eval_v<OUT>(ff.z);
            for (int i = 0; i < 3; ++i) q.a[i] = q.a[i] - q.f[i];
        } else {
            q.f[0] = q.f[1] = q.f[2] = T(0);
        }
        if (!valid) q.s = T(1);  // keep tau finite on idle lanes
        if constexpr (MAPPED)
            base_state_g(P, geo, q);
        else
            base_state(P, q);

        T X[4], Y[4][3];
        if constexpr (FUSED) {
            // the residual at this state, projected like the residual kernel's
            gp_residual_terms(P, q, X, Y);
            vec4<T> rr;
            if constexpr (MAPPED) {
                for (int c = 0; c < 4; ++c) {
                    const T y0 = Y[c][0], y1 = Y[c][1], y2 = Y[c][2];
                    Y[c][0] = geo.det * (geo.Ji[0][0] * y0 + geo.Ji[0][1] * y1 + geo.Ji[0][2] * y2);
                    Y[c][1] = geo.det * (geo.Ji[1][0] * y0 + geo.Ji[1][1] * y1 + geo.Ji[1][2] * y2);
                    Y[c][2] = geo.det * (geo.Ji[2][0] * y0 + geo.Ji[2][1] * y1 + geo.Ji[2][2] * y2);
                    X[c] = geo.det * X[c];
                }
                project2<OUT>(X[0], Y[0], X[1], Y[1], sx, sy, sz, rr.x, rr.y);
                project2<OUT>(X[2], Y[2], X[3], Y[3], sx, sy, sz, rr.z, rr.w);
            } else {
                project2<OUT>(X[0], Y[0], X[1], Y[1], sx, sy, sz, rr.x, rr.y);
                project2<OUT>(X[2], Y[2], X[3], Y[3], sx, sy, sz, rr.z, rr.w);
                rr.x = P.detJ * rr.x;
                rr.y = P.detJ * rr.y;
                rr.z = P.detJ * rr.z;
                rr.w = P.detJ * rr.w;
            }
            if (slot < nel) rel[rel_records(nel) + rel_at(nel, slot, g)] = valid ? rr : zero;
        }
        if (!JAC) {
            gp_residual_terms(P, q, X, Y);
        } else {
            vec4<T> xx = valid ? load_c<T>(P.x + node) : zero;
            // native FP64: the chain factor c_v scales the direction's
            // velocity at the node (3 multiplies instead of 12 at the Gauss
            // point), and da = (c_a / c_v) dv
            constexpr bool kNodeScale = std::is_same<T, double>::value;
            if constexpr (kNodeScale) {
                xx.x = P.c_v * xx.x;
                xx.y = P.c_v * xx.y;
                xx.z = P.c_v * xx.z;
            }
            T dv[3], dgv[3][3], da[3], dp, dgp[3];
            {
                VG<T> e0, e1, e2, e3;
                eval_vg4<OUT>(xx, sx, sy, sz, e0, e1, e2, e3);
                if constexpr (MAPPED) {
                    to_phys(geo, e0);
                    to_phys(geo, e1);
                    to_phys(geo, e2);
                    to_phys(geo, e3);
                }
                if constexpr (kNodeScale) {
                    dv[0] = e0.v; da[0] = P.c_av * e0.v;
                    dv[1] = e1.v; da[1] = P.c_av * e1.v;
                    dv[2] = e2.v; da[2] = P.c_av * e2.v;
                    dgv[0][0] = e0.gx; dgv[0][1] = e0.gy; dgv[0][2] = e0.gz;
                    dgv[1][0] = e1.gx; dgv[1][1] = e1.gy; dgv[1][2] = e1.gz;
                    dgv[2][0] = e2.gx; dgv[2][1] = e2.gy; dgv[2][2] = e2.gz;
                } else {
                    const T cv = P.c_v, ca = P.c_a;
                    dv[0] = cv * e0.v; da[0] = ca * e0.v;
                    dv[1] = cv * e1.v; da[1] = ca * e1.v;
                    dv[2] = cv * e2.v; da[2] = ca * e2.v;
                    dgv[0][0] = cv * e0.gx; dgv[0][1] = cv * e0.gy; dgv[0][2] = cv * e0.gz;
                    dgv[1][0] = cv * e1.gx; dgv[1][1] = cv * e1.gy; dgv[1][2] = cv * e1.gz;
                    dgv[2][0] = cv * e2.gx; dgv[2][1] = cv * e2.gy; dgv[2][2] = cv * e2.gz;
                }
                dp = e3.v; dgp[0] = e3.gx; dgp[1] = e3.gy; dgp[2] = e3.gz;
            }
            // d tau_M = -1/2 tau_M^3 s dQ with dQ = 2 v.G dv
            T vGdv, q0;
            if constexpr (MAPPED) {
                vGdv = vGdv_full(geo, q, dv);
                q0 = geo.q0;
            } else {
                vGdv = dot3_t(P.G0 * q.v[0], dv[0], P.G1 * q.v[1], dv[1], P.G2 * q.v[2], dv[2]);
                q0 = P.q0;
            }
            gp_jacobian_terms(P, q, dv, dgv, da, dp, dgp, vGdv, q0, X, Y);
        }
        vec4<T> r;
        if constexpr (MAPPED) {
            // grad N . Y = grad_xi N . (Ji Y); det J per Gauss point
            for (int c = 0; c < 4; ++c) {
                const T y0 = Y[c][0], y1 = Y[c][1], y2 = Y[c][2];
                Y[c][0] = geo.det * (geo.Ji[0][0] * y0 + geo.Ji[0][1] * y1 + geo.Ji[0][2] * y2);
                Y[c][1] = geo.det * (geo.Ji[1][0] * y0 + geo.Ji[1][1] * y1 + geo.Ji[1][2] * y2);
                Y[c][2] = geo.det * (geo.Ji[2][0] * y0 + geo.Ji[2][1] * y1 + geo.Ji[2][2] * y2);
                X[c] = geo.det * X[c];
            }
            project2<OUT>(X[0], Y[0], X[1], Y[1], sx, sy, sz, r.x, r.y);
            project2<OUT>(X[2], Y[2], X[3], Y[3], sx, sy, sz, r.z, r.w);
        } else {
            project2<OUT>(X[0], Y[0], X[1], Y[1], sx, sy, sz, r.x, r.y);
            project2<OUT>(X[2], Y[2], X[3], Y[3], sx, sy, sz, r.z, r.w);
            r.x = P.detJ * r.x;
            r.y = P.detJ * r.y;
            r.z = P.detJ * r.z;
            r.w = P.detJ * r.w;
        }
        if (slot < nel) rel[rel_at(nel, slot, g)] = valid ? r : zero;
    }
    __syncthreads();

    // Node block of the brick: each node sums the contributions of the (up to
    // 8) brick elements around it, corner by corner in a fixed order.
    const int nx1 = P.bx + 1, ny1 = P.by + 1, nz1 = P.bz + 1;
    const int nnodes = nx1 * ny1 * nz1;
    constexpr int kOut = FUSED ? 2 : 1;
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
        vec4<T> *blk = (o ? P.blocks2 : P.blocks) + (size_t)brick * nnodes;
        const vec4<T> *rl = rel + o * rel_records(nel);
        for (int nl = threadIdx.x; nl < nnodes; nl += blockDim.x) {
            const int ix = nl % nx1, iy = (nl / nx1) % ny1, iz = nl / (nx1 * ny1);
            vec4<T> acc = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int lx = ix - (c & 1), ly = iy - ((c >> 1) & 1), lz = iz - ((c >> 2) & 1);
                if (lx < 0 || ly < 0 || lz < 0 || lx >= P.bx || ly >= P.by || lz >= P.bz) continue;
                const vec4<T> r = rl[rel_at(nel, (lz * P.by + ly) * P.bx + lx, c)];
                acc.x += r.x;
                acc.y += r.y;
                acc.z += r.z;
                acc.w += r.w;
            }
            blk[nl] = acc;
        }
    }
}

// Candidate (brick, local index) pairs of node coordinate i along one axis,
// lower brick first.
static __device__ __forceinline__ int axis_candidates(int i, int b, int nb, int *cb, int *cl)
{
    int k = 0;
    const int q = i / b, r = i - q * b;
    if (r == 0 && q > 0) {
        cb[k] = q - 1;
        cl[k] = b;
        ++k;
    }
    if (q < nb) {
        cb[k] = q;
        cl[k] = r;
        ++k;
    }
    return k;
}

// Sum, for one node, the (up to 8) brick node blocks that contain it, lower
// bricks first (FUSED: the residual's blocks into out2 as well).
template <typename T, bool FUSED = false>
__device__ __forceinline__ void gather_node(const VmsArgs<T> &P, int node)
{
    using S = typename StorageOf<T>::type;
    const int NX1 = P.Nx + 1, NY1 = P.Ny + 1;
    const int nx1 = P.bx + 1, ny1 = P.by + 1, nz1 = P.bz + 1;
    const int nnodes = nx1 * ny1 * nz1;
    {
        const int i = node % NX1, j = (node / NX1) % NY1, k = node / (NX1 * NY1);
        int cbx[2], clx[2], cby[2], cly[2], cbz[2], clz[2];
        const int kx = axis_candidates(i, P.bx, P.nbx, cbx, clx);
        const int ky = axis_candidates(j, P.by, P.nby, cby, cly);
        const int kz = axis_candidates(k, P.bz, P.nbz, cbz, clz);
        constexpr int kOut = FUSED ? 2 : 1;
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const vec4<T> *blocks = o ? P.blocks2 : P.blocks;
            vec4<T> acc = {T(0), T(0), T(0), T(0)};
            for (int c = 0; c < kz; ++c)
                for (int b = 0; b < ky; ++b)
                    for (int a = 0; a < kx; ++a) {
                        const size_t brick = cbx[a] + P.nbx * (cby[b] + (size_t)P.nby * cbz[c]);
                        const int nl = clx[a] + nx1 * (cly[b] + ny1 * clz[c]);
                        const vec4<T> r = ld4_blk(blocks + brick * nnodes + nl);
                        acc.x += r.x;
                        acc.y += r.y;
                        acc.z += r.z;
                        acc.w += r.w;
                    }
            (o ? P.out2 : P.out)[node] = {to_s(acc.x), to_s(acc.y), to_s(acc.z), to_s(acc.w)};
        }
    }
}

template <typename T>
VmsArgs<T> make_args(const fsi_mesh *m, const Brick &b, const void *U, const void *A,
                     const void *f, const void *x, void *out)
{
    VmsArgs<T> P;
    P.Nx = m->grid.N[0];
    P.Ny = m->grid.N[1];
    P.Nz = m->grid.N[2];
    P.bx = b.bx;
    P.by = b.by;
    P.bz = b.bz;
    P.nbx = (P.Nx + b.bx - 1) / b.bx;
    P.nby = (P.Ny + b.by - 1) / b.by;
    P.nbz = (P.Nz + b.bz - 1) / b.bz;
    const double rho = m->phys.rho, mu = m->phys.mu, dt = m->phys.dt;
    const double *h = m->grid.h;
    double G[3], trG = 0.0, GG = 0.0;
    for (int k = 0; k < 3; ++k) {
        G[k] = 4.0 / (h[k] * h[k]);
        trG += G[k];
        GG += G[k] * G[k];
    }
    const double nu = mu / rho;
    P.rho = (T)rho;
    P.mu = (T)mu;
    P.inv_rho = (T)(1.0 / rho);
    P.G0 = (T)G[0];
    P.G1 = (T)G[1];
    P.G2 = (T)G[2];
    P.inv_trG = (T)(1.0 / trG);
    P.q0 = (T)(m->phys.C_T / (dt * dt) + m->phys.C_I * nu * nu * GG);
    P.ih0 = (T)(1.0 / h[0]);
    P.ih1 = (T)(1.0 / h[1]);
    P.ih2 = (T)(1.0 / h[2]);
    P.detJ = (T)(h[0] * h[1] * h[2] / 8.0);
    P.c_a = (T)m->alpha_m;
    P.c_v = (T)(m->alpha_f * m->gamma * dt);
    P.c_av = (T)(m->alpha_m / (m->alpha_f * m->gamma * dt));
    P.ct_dt2 = (T)(m->phys.C_T / (dt * dt));
    P.CInu2 = (T)(m->phys.C_I * nu * nu);
    P.has_s = m->phys.has_s != 0;
    using S = typename StorageOf<T>::type;
    P.Xc = (const vec4<S> *)(sizeof(S) == 8 ? m->coords64 : m->coords32);
    P.geo = nullptr;
    P.U = (const vec4<S> *)U;
    P.A = (const vec4<S> *)A;
    P.f = (const vec4<S> *)f;
    P.x = (const vec4<S> *)x;
    P.blocks = (vec4<T> *)m->vms_scratch;
    P.out = (vec4<S> *)out;
    P.blocks2 = nullptr;
    P.out2 = nullptr;
    return P;
}

}  // namespace vmsd
}  // namespace fsi
