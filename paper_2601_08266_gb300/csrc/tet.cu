// tet.cu -- the hot path on unstructured meshes of linear tetrahedra (P1-P1,
// the element family of the paper's valve fluid mesh, Sec. 4): VMS residual
// and Jacobian apply (Sec. 2.1, 2.4), point location, interpolation and
// spreading (Sec. 2.3).
//
// VMS operators.  Four consecutive lanes own one tetrahedron: lane a first
// loads node a of the element (fields and coordinates) and then acts as
// quadrature point a of the symmetric 4-point rule (barycentric coordinates
// al at node a, be elsewhere).  The element geometry (J = [x1-x0, x2-x0,
// x3-x0], J^-1, the metric G = J^-T J^-1 of Sec. 2.1, G:G, 1/tr G, the weight)
// is a per-element table computed once per compute type (the mesh does not
// move; reading 72-144 B per element costs less than forming it in every
// lane of every apply); P1 gradients are constant per
// element, so a field's gradient is the group sum of u_a grad N_a and its
// value at point q is be * sum_a u_a + (al - be) u_q.  The Gauss-point
// algebra is the one the hexahedral kernels use (gp_residual_terms /
// gp_jacobian_terms with the full metric).  The projection onto test
// function a is w (be sum_q X_q + (al - be) X_a + grad N_a . sum_q Y_q) with
// w = |det J| / 24.  Each lane writes its node's contribution into a per-slot
// scratch [E][4]; a gather kernel sums, for every node, its slots in a fixed
// order (node -> slot lists built once at creation), so the result is
// deterministic and atomic-free.
//
// Location.  A uniform bucket grid over the mesh's bounding box lists, in
// increasing element order, the elements whose (padded) bounding box meets
// each bucket.  A point tests the candidates of its bucket in that order:
// an FP32 barycentric test discards elements it is clearly outside of (and
// stops the scan at one it is almost surely inside of), and the FP64
// barycentric coordinates, evaluated with round-to-nearest
// operations in the same order as the definition (no contraction), decide:
// the first element whose four coordinates are all >= -1e-12 holds the
// point.  That is the first element in element order, as a search over all
// elements would find.  The cell table (element -> points) is the stable
// counting sort of the grid path.
//
// Spreading.  Per element, four lanes sum the barycentric corner
// contributions w_B N_a(lam_B) lambda_B over the element's points (perm
// order, strided by lane), a fixed two-level transpose-reduce gives the 12
// corner sums; then every node sums the corner sums of its occupied elements
// in slot order.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "fsi_internal.cuh"
#include "vms_device.cuh"

struct fsi_tetmesh {
    int device;
    cudaStream_t stream;
    int64_t n_nodes, n_elems;
    fsi_physics phys;
    double alpha_m, alpha_f, gamma;
    double4 *X64;
    float4 *X32;
    int4 *tets;
    int32_t *node_start, *node_slot;  // node -> slots e*4 + corner, increasing
    // location buckets
    int nb[3];
    double lo[3], inv_cell[3], box_lo[3], box_hi[3];
    int32_t *bucket_start, *bucket_tets;
    // scratch
    void *slot_scratch;    // [E][4] vec4 in the compute type (32 B per slot)
    void *corner_scratch;  // [E][4][3] spreading corner sums (8 B per value)
    int32_t *fill;         // [E+1]
    int32_t *scan_tmp;
    unsigned long long *nout;
    // distance-2 node colouring for probing the nodal diagonal blocks
    int32_t *colors;
    int n_colors;
    // per-element geometry (J^-1, G, G:G, 1/tr G, |det J|/24) in each compute
    // type [FSI_F64, FSI_F32, FSI_DF64], computed on first use
    void *geo[3];
};

namespace fsi {
namespace {

using namespace vmsd;

constexpr double kTetAl = 0.58541019662496845446;  // (5 + 3 sqrt 5) / 20
constexpr double kTetBe = 0.13819660112501051518;  // (5 - sqrt 5) / 20

template <typename T> __device__ __forceinline__ T tet_al();
template <typename T> __device__ __forceinline__ T tet_be();
template <> __device__ __forceinline__ double tet_al<double>() { return kTetAl; }
template <> __device__ __forceinline__ double tet_be<double>() { return kTetBe; }
template <> __device__ __forceinline__ float tet_al<float>() { return (float)kTetAl; }
template <> __device__ __forceinline__ float tet_be<float>() { return (float)kTetBe; }
constexpr float kTetAlH = static_cast<float>(kTetAl);
constexpr float kTetAlL = static_cast<float>(kTetAl - static_cast<double>(kTetAlH));
constexpr float kTetBeH = static_cast<float>(kTetBe);
constexpr float kTetBeL = static_cast<float>(kTetBe - static_cast<double>(kTetBeH));
template <> __device__ __forceinline__ df64 tet_al<df64>() { return df64(kTetAlH, kTetAlL); }
template <> __device__ __forceinline__ df64 tet_be<df64>() { return df64(kTetBeH, kTetBeL); }

// sum over the group of four lanes (butterfly; every lane gets the same value)
template <typename T> __device__ __forceinline__ T group_sum(T v)
{
    v = v + shx(v, 1);
    return v + shx(v, 2);
}

template <typename T> __device__ __forceinline__ T abs_t(T v) { return v < T(0) ? -v : v; }
template <> __device__ __forceinline__ df64 abs_t<df64>(df64 v) { return v.hi < 0.0f ? -v : v; }

// Element geometry from the four corner coordinates c[b][i]: J[i][k] =
// c[k+1][i] - c[0][i], J^-1 by cofactors, G = J^-T J^-1, G:G, 1/tr G and
// the quadrature weight |det J| / 24; it fills the per-element geometry table
// that the VMS kernels read.
constexpr int kTetGeo = 18;  // Ji[9], G00 G01 G02 G11 G12 G22, G:G, 1/trG, w

template <typename T> __device__ __forceinline__ void tet_geometry(const T (&c)[4][3], T (&out)[kTetGeo])
{
    T J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) J[i][k] = c[k + 1][i] - c[0][i];
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
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            G[i][j] = dot3_t(Ji[0][i], Ji[0][j], Ji[1][i], Ji[1][j], Ji[2][i], Ji[2][j]);
            GG = fma_t(G[i][j], G[i][j], GG);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * i + k] = Ji[i][k];
    out[9] = G[0][0];
    out[10] = G[0][1];
    out[11] = G[0][2];
    out[12] = G[1][1];
    out[13] = G[1][2];
    out[14] = G[2][2];
    out[15] = GG;
    out[16] = inv_t(G[0][0] + G[1][1] + G[2][2]);
    out[17] = abs_t(det) * T(1.0 / 24.0);
}

template <typename T>
__global__ void tet_geo_kernel(int64_t E, const int4 *__restrict__ tets,
                               const vec4<typename StorageOf<T>::type> *__restrict__ X,
                               T *__restrict__ geo)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int4 t = tets[e];
        const int nd[4] = {t.x, t.y, t.z, t.w};
        T c[4][3];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const vec4<T> x = load_c<T>(X + nd[b]);
            c[b][0] = x.x;
            c[b][1] = x.y;
            c[b][2] = x.z;
        }
        T g[kTetGeo];
        tet_geometry(c, g);
#pragma unroll
        for (int k = 0; k < kTetGeo; ++k) geo[e * kTetGeo + k] = g[k];
    }
}

template <typename T> struct TetArgs {
    using S = typename StorageOf<T>::type;
    VmsArgs<T> V;  // physics, chain factors and the field pointers U, A, f, x
    int64_t E;
    const vec4<S> *X;
    const int4 *tets;
    const T *geo;  // [E][kTetGeo]
    vec4<T> *slots;
};

template <typename T, bool JAC> __global__ void __launch_bounds__(256) tet_vms_kernel(TetArgs<T> P)
{
    using S = typename StorageOf<T>::type;
    const VmsArgs<T> &V = P.V;
    const int a = threadIdx.x & 3;
    const int lane = threadIdx.x & 31;
    // warp-uniform trip count: every lane of a warp shuffles in every pass
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t - lane < 4 * P.E;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t >> 2;
        const bool valid = e < P.E;
        const vec4<T> zero = {T(0), T(0), T(0), T(0)};
        int node = 0;
        if (valid) {
            const int4 tt = P.tets[e];
            node = a == 0 ? tt.x : (a == 1 ? tt.y : (a == 2 ? tt.z : tt.w));
        }
        const vec4<T> u = valid ? load_c<T>(V.U + node) : zero;
        const vec4<T> ac = valid ? load_c<T>(V.A + node) : zero;
        const vec4<T> ff = (valid && V.f) ? load_c<T>(V.f + node) : zero;

        // element geometry from the table (idle lanes: the unit reference
        // tetrahedron, J = I)
        Geo<T> geo;
        T GG;
        if (valid) {
            const T *g = P.geo + e * kTetGeo;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) geo.Ji[i][k] = g[3 * i + k];
            geo.G[0][0] = g[9];
            geo.G[0][1] = geo.G[1][0] = g[10];
            geo.G[0][2] = geo.G[2][0] = g[11];
            geo.G[1][1] = g[12];
            geo.G[1][2] = geo.G[2][1] = g[13];
            geo.G[2][2] = g[14];
            GG = g[15];
            geo.inv_trG = g[16];
            geo.det = g[17];  // holds the quadrature weight |det J| / 24
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) geo.Ji[i][k] = geo.G[i][k] = T(i == k ? 1 : 0);
            GG = T(3);
            geo.inv_trG = inv_t(T(3));
            geo.det = T(1.0 / 24.0);
        }
        geo.q0 = fma_t(V.CInu2, GG, V.ct_dt2);
        // grad N of this lane's node
        T dN[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T s3 = -(geo.Ji[0][j] + geo.Ji[1][j] + geo.Ji[2][j]);
            dN[j] = a == 0 ? s3 : (a == 1 ? geo.Ji[0][j] : (a == 2 ? geo.Ji[1][j] : geo.Ji[2][j]));
        }
        const T al = tet_al<T>(), be = tet_be<T>(), amb = al - be;
        // Values and gradients of two fields at a time: float and double-float
        // pairs run on the paired FP32 instructions (the double-float pair is
        // bit-identical to the scalar sequence); double pairs are two scalars.
        using PO = PairOf<T>;
        using PT = typename PO::type;
        const PT amb2 = PO::pack(amb, amb), be2 = PO::pack(be, be);
        PT dN2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) dN2[j] = PO::pack(dN[j], dN[j]);
        auto value = [&](T w) { return fma_t(amb, w, be * group_sum(w)); };
        auto value2 = [&](T w1, T w2, T &r1, T &r2) {
            const PT w = PO::pack(w1, w2);
            const PT r = fma_t(amb2, w, be2 * group_sum(w));
            r1 = PO::first(r);
            r2 = PO::second(r);
        };
        auto grad2 = [&](T w1, T w2, T (&g1)[3], T (&g2)[3]) {
            const PT w = PO::pack(w1, w2);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const PT gs = group_sum(w * dN2[j]);
                g1[j] = PO::first(gs);
                g2[j] = PO::second(gs);
            }
        };

        GP<T> q;
        {
            value2(u.x, u.y, q.v[0], q.v[1]);
            value2(u.z, u.w, q.v[2], q.p);
            grad2(u.x, u.y, q.gv[0], q.gv[1]);
            grad2(u.z, u.w, q.gv[2], q.gp);
            T sv;
            value2(ac.x, ac.y, q.a[0], q.a[1]);
            value2(ac.z, ac.w, q.a[2], sv);
            q.s = V.has_s ? sv : T(1);
            if (V.f) {
                value2(ff.x, ff.y, q.f[0], q.f[1]);
                q.f[2] = value(ff.z);
                for (int i = 0; i < 3; ++i) q.a[i] = q.a[i] - q.f[i];
            } else {
                q.f[0] = q.f[1] = q.f[2] = T(0);
            }
            if (!valid) q.s = T(1);
        }
        base_state_g(V, geo, q);

        T X[4], Y[4][3];
        if (!JAC) {
            gp_residual_terms(V, q, X, Y);
        } else {
            const vec4<T> xx = valid ? load_c<T>(V.x + node) : zero;
            T val[3], dp, g[3][3], dgp[3];
            value2(xx.x, xx.y, val[0], val[1]);
            value2(xx.z, xx.w, val[2], dp);
            grad2(xx.x, xx.y, g[0], g[1]);
            grad2(xx.z, xx.w, g[2], dgp);
            T dv[3], da[3], dgv[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dv[i] = V.c_v * val[i];
                da[i] = V.c_a * val[i];
#pragma unroll
                for (int j = 0; j < 3; ++j) dgv[i][j] = V.c_v * g[i][j];
            }
            const T vGdv = vGdv_full(geo, q, dv);
            gp_jacobian_terms(V, q, dv, dgv, da, dp, dgp, vGdv, geo.q0, X, Y);
        }
        // projection onto this lane's test function, two components at a time
        const PT w2 = PO::pack(geo.det, geo.det);
        T r[4];
#pragma unroll
        for (int cc = 0; cc < 4; cc += 2) {
            const PT Xp = PO::pack(X[cc], X[cc + 1]);
            const PT gx = group_sum(PO::pack(Y[cc][0], Y[cc + 1][0]));
            const PT gy = group_sum(PO::pack(Y[cc][1], Y[cc + 1][1]));
            const PT gz = group_sum(PO::pack(Y[cc][2], Y[cc + 1][2]));
            const PT t0 = fma_t(amb2, Xp, be2 * group_sum(Xp));
            const PT rr = w2 * (t0 + dot3_t(dN2[0], gx, dN2[1], gy, dN2[2], gz));
            r[cc] = PO::first(rr);
            r[cc + 1] = PO::second(rr);
        }
        if (valid) P.slots[t] = vec4<T>{r[0], r[1], r[2], r[3]};
    }
}

template <typename T>
__global__ void tet_gather_kernel(int64_t n, const int32_t *__restrict__ start,
                                  const int32_t *__restrict__ slot, const vec4<T> *__restrict__ in,
                                  vec4<typename StorageOf<T>::type> *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vec4<T> acc = {T(0), T(0), T(0), T(0)};
        for (int k = start[i]; k < start[i + 1]; ++k) {
            const vec4<T> r = ld4_blk(in + slot[k]);
            acc.x += r.x;
            acc.y += r.y;
            acc.z += r.z;
            acc.w += r.w;
        }
        out[i] = {to_s(acc.x), to_s(acc.y), to_s(acc.z), to_s(acc.w)};
    }
}

// ------------------------------------------------------------------ location
struct BucketArgs {
    int nb[3];
    double lo[3], inv_cell[3], box_lo[3], box_hi[3];
};

// barycentric coordinates, round-to-nearest operations in the order of the
// definition (e_k = x_k - x_0, d = P - x_0, D = e1.(e2 x e3), ...)
__device__ __forceinline__ void barycentric64(const double4 &x0, const double4 &x1,
                                              const double4 &x2, const double4 &x3,
                                              const double P[3], double lam[4])
{
    const double e1[3] = {__dsub_rn(x1.x, x0.x), __dsub_rn(x1.y, x0.y), __dsub_rn(x1.z, x0.z)};
    const double e2[3] = {__dsub_rn(x2.x, x0.x), __dsub_rn(x2.y, x0.y), __dsub_rn(x2.z, x0.z)};
    const double e3[3] = {__dsub_rn(x3.x, x0.x), __dsub_rn(x3.y, x0.y), __dsub_rn(x3.z, x0.z)};
    const double d[3] = {__dsub_rn(P[0], x0.x), __dsub_rn(P[1], x0.y), __dsub_rn(P[2], x0.z)};
    auto cross = [](const double *u, const double *v, double *w) {
        w[0] = __dsub_rn(__dmul_rn(u[1], v[2]), __dmul_rn(u[2], v[1]));
        w[1] = __dsub_rn(__dmul_rn(u[2], v[0]), __dmul_rn(u[0], v[2]));
        w[2] = __dsub_rn(__dmul_rn(u[0], v[1]), __dmul_rn(u[1], v[0]));
    };
    auto dot = [](const double *u, const double *v) {
        return __dadd_rn(__dadd_rn(__dmul_rn(u[0], v[0]), __dmul_rn(u[1], v[1])),
                         __dmul_rn(u[2], v[2]));
    };
    double c[3], a[3], b[3];
    cross(e2, e3, c);
    const double D = dot(e1, c);
    const double l1 = __ddiv_rn(dot(d, c), D);
    cross(d, e3, a);
    const double l2 = __ddiv_rn(dot(e1, a), D);
    cross(e2, d, b);
    const double l3 = __ddiv_rn(dot(e1, b), D);
    lam[1] = l1;
    lam[2] = l2;
    lam[3] = l3;
    lam[0] = __dsub_rn(__dsub_rn(__dsub_rn(1.0, l1), l2), l3);
}

// FP32 screen: 0 where the point is clearly outside (some barycentric
// coordinate below -1e-2), 2 where it is almost surely inside (all above
// -1e-5), 1 in between
__device__ __forceinline__ int screen32(const float4 &x0, const float4 &x1, const float4 &x2,
                                        const float4 &x3, const float P[3])
{
    const float e1[3] = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
    const float e2[3] = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
    const float e3[3] = {x3.x - x0.x, x3.y - x0.y, x3.z - x0.z};
    const float d[3] = {P[0] - x0.x, P[1] - x0.y, P[2] - x0.z};
    const float c0 = e2[1] * e3[2] - e2[2] * e3[1], c1 = e2[2] * e3[0] - e2[0] * e3[2],
                c2 = e2[0] * e3[1] - e2[1] * e3[0];
    const float D = e1[0] * c0 + e1[1] * c1 + e1[2] * c2;
    const float iD = 1.0f / D;
    const float l1 = (d[0] * c0 + d[1] * c1 + d[2] * c2) * iD;
    const float a0 = d[1] * e3[2] - d[2] * e3[1], a1 = d[2] * e3[0] - d[0] * e3[2],
                a2 = d[0] * e3[1] - d[1] * e3[0];
    const float l2 = (e1[0] * a0 + e1[1] * a1 + e1[2] * a2) * iD;
    const float b0 = e2[1] * d[2] - e2[2] * d[1], b1 = e2[2] * d[0] - e2[0] * d[2],
                b2 = e2[0] * d[1] - e2[1] * d[0];
    const float l3 = (e1[0] * b0 + e1[1] * b1 + e1[2] * b2) * iD;
    const float l0 = 1.0f - l1 - l2 - l3;
    const float lmin = fminf(fminf(l0, l1), fminf(l2, l3));
    if (lmin < -1e-2f) return 0;  // (a NaN falls through to the exact test)
    return lmin >= -1e-5f ? 2 : 1;
}

__global__ void tet_locate_kernel(int64_t m, BucketArgs B, const double4 *__restrict__ X64,
                                  const float4 *__restrict__ X32, const int4 *__restrict__ tets,
                                  const int32_t *__restrict__ bstart,
                                  const int32_t *__restrict__ btets, const double *__restrict__ P,
                                  int32_t *__restrict__ elem, double *__restrict__ lam_out,
                                  int32_t *__restrict__ count, unsigned long long *n_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double p[3] = {P[3 * i], P[3 * i + 1], P[3 * i + 2]};
        int found = -1;
        double lam[4] = {0.0, 0.0, 0.0, 0.0};
        bool inbox = true;
        for (int k = 0; k < 3; ++k)
            inbox = inbox && p[k] >= B.box_lo[k] && p[k] <= B.box_hi[k];  // NaN: outside
        if (inbox) {
            int bi[3];
            for (int k = 0; k < 3; ++k) {
                int v = (int)floor((p[k] - B.lo[k]) * B.inv_cell[k]);
                bi[k] = v < 0 ? 0 : (v >= B.nb[k] ? B.nb[k] - 1 : v);
            }
            const int64_t bk = bi[0] + (int64_t)B.nb[0] * (bi[1] + (int64_t)B.nb[1] * bi[2]);
            const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
            // the FP32 screen collects candidates in list order (up to four,
            // or up to one it finds almost surely inside), then the exact FP64
            // test runs on them in that order; the lanes of a warp reach the
            // FP64 block together far more often than if each ran it at its
            // own position in the list
            int c = bstart[bk];
            const int cend = bstart[bk + 1];
            while (c < cend && found < 0) {
                int cand[4], nc = 0;
                bool likely = false;
                for (; c < cend && nc < 4 && !likely; ++c) {
                    const int e = btets[c];
                    const int4 t = tets[e];
                    const int sc = screen32(X32[t.x], X32[t.y], X32[t.z], X32[t.w], pf);
                    if (sc > 0) cand[nc++] = e;
                    likely = sc == 2;
                }
                for (int k = 0; k < nc; ++k) {
                    const int4 t = tets[cand[k]];
                    barycentric64(X64[t.x], X64[t.y], X64[t.z], X64[t.w], p, lam);
                    if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 &&
                        lam[3] >= -1e-12) {
                        found = cand[k];
                        break;
                    }
                }
            }
        }
        if (found < 0) {
            elem[i] = -1;
            lam_out[3 * i] = lam_out[3 * i + 1] = lam_out[3 * i + 2] = 0.0;
            atomicAdd(n_out, 1ull);
            continue;
        }
        elem[i] = found;
        lam_out[3 * i] = lam[1];
        lam_out[3 * i + 1] = lam[2];
        lam_out[3 * i + 2] = lam[3];
        if (count) atomicAdd(count + found, 1);
    }
}

// ------------------------------------------------------------ interp / spread
template <typename T, typename S = typename StorageOf<T>::type>
__global__ void tet_interp_kernel(int64_t m, int64_t E, const int4 *__restrict__ tets,
                                  const int32_t *__restrict__ elem, const S *__restrict__ lam,
                                  const vec4<S> *__restrict__ U, S *__restrict__ u)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int e = elem[b];
        T ux = T(0), uy = T(0), uz = T(0);
        if (e >= 0 && e < E) {
            const int4 t = tets[e];
            const T l1 = to_c<T>(lam[3 * b]), l2 = to_c<T>(lam[3 * b + 1]),
                    l3 = to_c<T>(lam[3 * b + 2]);
            const T Nv[4] = {T(1) - l1 - l2 - l3, l1, l2, l3};
            const int nd[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const auto v = ld4(U + nd[a]);
                ux = madd(Nv[a], to_c<T>(v.x), ux);
                uy = madd(Nv[a], to_c<T>(v.y), uy);
                uz = madd(Nv[a], to_c<T>(v.z), uz);
            }
        }
        u[3 * b] = to_s(ux);
        u[3 * b + 1] = to_s(uy);
        u[3 * b + 2] = to_s(uz);
    }
}

// corner sums S[e][4][3] of the points of each element: a warp takes 8
// elements, four lanes per element; lane k sums the element's points k, k+4,
// ... in perm order, then a two-level transpose-reduce leaves corner 2 b1 + b0
// (3 values) in the lane with bits (b1, b0)
template <typename T, typename S = typename StorageOf<T>::type>
__global__ void tet_spread_cells_kernel(int64_t E, const S *__restrict__ lam,
                                        const int32_t *__restrict__ start,
                                        const int32_t *__restrict__ perm,
                                        const S *__restrict__ lamv, const S *__restrict__ w,
                                        T *__restrict__ Ssum)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e0 = warp * 8; e0 < E; e0 += nwarps * 8) {
        const int64_t e = e0 + (lane >> 2);
        int lo = 0, hi = 0;
        if (e < E) {
            lo = start[e];
            hi = start[e + 1];
        }
        if (__all_sync(0xffffffffu, hi == lo)) continue;
        T acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = T(0);
        for (int p = lo + (lane & 3); p < hi; p += 4) {
            const int b = perm[p];
            const T l1 = to_c<T>(lam[3 * b]), l2 = to_c<T>(lam[3 * b + 1]),
                    l3 = to_c<T>(lam[3 * b + 2]);
            const T s = w ? to_c<T>(w[b]) : T(1);
            const T Nv[4] = {(T(1) - l1 - l2 - l3) * s, l1 * s, l2 * s, l3 * s};
            const T f0 = to_c<T>(lamv[3 * b]), f1 = to_c<T>(lamv[3 * b + 1]),
                    f2 = to_c<T>(lamv[3 * b + 2]);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                acc[3 * a] = madd(Nv[a], f0, acc[3 * a]);
                acc[3 * a + 1] = madd(Nv[a], f1, acc[3 * a + 1]);
                acc[3 * a + 2] = madd(Nv[a], f2, acc[3 * a + 2]);
            }
        }
        const bool b1 = lane & 2, b0 = lane & 1;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T send = b1 ? acc[k] : acc[6 + k];
            const T keep = b1 ? acc[6 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 2);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T send = b0 ? acc[k] : acc[3 + k];
            const T keep = b0 ? acc[3 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 1);
        }
        if (hi > lo) {
            T *dst = Ssum + e * 12 + (b1 ? 6 : 0) + (b0 ? 3 : 0);
            dst[0] = acc[0];
            dst[1] = acc[1];
            dst[2] = acc[2];
        }
    }
}

template <typename T, typename S = typename StorageOf<T>::type>
__global__ void tet_spread_nodes_kernel(int64_t n, const int32_t *__restrict__ nstart,
                                        const int32_t *__restrict__ nslot,
                                        const int32_t *__restrict__ start,
                                        const T *__restrict__ Ssum, S *__restrict__ F,
                                        int accumulate)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T fx = T(0), fy = T(0), fz = T(0);
        for (int k = nstart[i]; k < nstart[i + 1]; ++k) {
            const int sl = nslot[k];
            const int e = sl >> 2;
            if (start[e + 1] == start[e]) continue;
            const T *src = Ssum + (int64_t)e * 12 + 3 * (sl & 3);
            fx += src[0];
            fy += src[1];
            fz += src[2];
        }
        if (accumulate) {
            F[4 * i] = to_s(to_c<T>(F[4 * i]) + fx);
            F[4 * i + 1] = to_s(to_c<T>(F[4 * i + 1]) + fy);
            F[4 * i + 2] = to_s(to_c<T>(F[4 * i + 2]) + fz);
        } else {
            F[4 * i] = to_s(fx);
            F[4 * i + 1] = to_s(fy);
            F[4 * i + 2] = to_s(fz);
        }
    }
}

__global__ void pad_tet_coords_kernel(int64_t n, const double *X, double4 *X64, float4 *X32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
        X64[i] = make_double4(x, y, z, 0.0);
        X32[i] = make_float4((float)x, (float)y, (float)z, 0.0f);
    }
}

int grid_for(int64_t n, int threads, int cap = sm_count() * 32)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

fsi_status validate_tetmesh(const fsi_tetmesh *m)
{
    if (!m) return set_error(FSI_ERR_ARG, "tet mesh is NULL");
    return FSI_OK;
}

template <typename T>
TetArgs<T> tet_args(fsi_tetmesh *m, const void *U, const void *A, const void *f, const void *x)
{
    using S = typename StorageOf<T>::type;
    TetArgs<T> P;
    memset((void *)&P.V, 0, sizeof P.V);
    const double rho = m->phys.rho, mu = m->phys.mu, dt = m->phys.dt, nu = mu / rho;
    P.V.rho = T(rho);
    P.V.mu = T(mu);
    P.V.inv_rho = T(1.0 / rho);
    P.V.c_a = T(m->alpha_m);
    P.V.c_v = T(m->alpha_f * m->gamma * dt);
    P.V.ct_dt2 = T(m->phys.C_T / (dt * dt));
    P.V.CInu2 = T(m->phys.C_I * nu * nu);
    P.V.has_s = m->phys.has_s != 0;
    P.V.U = (const vec4<S> *)U;
    P.V.A = (const vec4<S> *)A;
    P.V.f = (const vec4<S> *)f;
    P.V.x = (const vec4<S> *)x;
    P.E = m->n_elems;
    P.X = (const vec4<S> *)(sizeof(S) == 8 ? (const void *)m->X64 : (const void *)m->X32);
    P.tets = m->tets;
    P.slots = (vec4<T> *)m->slot_scratch;
    return P;
}

template <typename T> constexpr int geo_slot()
{
    return std::is_same<T, double>::value ? 0 : (std::is_same<T, float>::value ? 1 : 2);
}

// the per-element geometry table of compute type T, built on first use
template <typename T> fsi_status ensure_geo(fsi_tetmesh *m)
{
    using S = typename StorageOf<T>::type;
    void *&g = m->geo[geo_slot<T>()];
    if (g) return FSI_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FSI_CUDA(cudaStreamIsCapturing(m->stream, &cap), "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return set_error(FSI_ERR_ARG, "tetrahedral geometry table: first apply of this compute "
                                      "type inside a stream capture");
    if (cudaMalloc(&g, (size_t)m->n_elems * kTetGeo * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        g = nullptr;
        return set_error(FSI_ERR_OOM, "tetrahedral geometry table: cudaMalloc failed");
    }
    const vec4<S> *X = (const vec4<S> *)(sizeof(S) == 8 ? (const void *)m->X64
                                                         : (const void *)m->X32);
    tet_geo_kernel<T><<<grid_for(m->n_elems, 256), 256, 0, m->stream>>>(m->n_elems, m->tets, X,
                                                                        (T *)g);
    return check_launch("tet geometry kernel");
}

template <typename T, bool JAC>
fsi_status tet_vms(fsi_tetmesh *m, const void *U, const void *A, const void *f, const void *x,
                   void *out)
{
    using S = typename StorageOf<T>::type;
    FSI_TRY(ensure_geo<T>(m));
    TetArgs<T> P = tet_args<T>(m, U, A, f, x);
    P.geo = (const T *)m->geo[geo_slot<T>()];
    const int64_t threads = 4 * m->n_elems;
    tet_vms_kernel<T, JAC><<<grid_for(threads, 256, sm_count() * 64), 256, 0, m->stream>>>(P);
    FSI_TRY(check_launch("tet vms kernel"));
    tet_gather_kernel<T><<<grid_for(m->n_nodes, 256), 256, 0, m->stream>>>(
        m->n_nodes, m->node_start, m->node_slot, P.slots, (vec4<S> *)out);
    return check_launch("tet gather kernel");
}

}  // namespace

void tet_set_stream(fsi_tetmesh *t, cudaStream_t s) { t->stream = s; }

void tet_set_physics(fsi_tetmesh *t, const fsi_physics *p)
{
    t->phys = *p;
    const double r = p->rho_inf;
    t->alpha_m = 0.5 * (3.0 - r) / (1.0 + r);
    t->alpha_f = 1.0 / (1.0 + r);
    t->gamma = 0.5 + t->alpha_m - t->alpha_f;
}

const int32_t *tet_colors(const fsi_tetmesh *t, int *n_colors)
{
    *n_colors = t->n_colors;
    return t->colors;
}

fsi_status tet_download(fsi_tetmesh *t, std::vector<double> &X, std::vector<int32_t> &tets,
                        double box_lo[3], double box_hi[3])
{
    std::vector<double4> x4((size_t)t->n_nodes);
    tets.resize((size_t)t->n_elems * 4);
    FSI_CUDA(cudaMemcpyAsync(x4.data(), t->X64, x4.size() * sizeof(double4), cudaMemcpyDeviceToHost,
                             t->stream),
             "memcpy");
    FSI_CUDA(cudaMemcpyAsync(tets.data(), t->tets, tets.size() * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, t->stream),
             "memcpy");
    FSI_CUDA(cudaStreamSynchronize(t->stream), "sync");
    X.resize((size_t)t->n_nodes * 3);
    for (int k = 0; k < 3; ++k) {
        box_lo[k] = INFINITY;
        box_hi[k] = -INFINITY;
    }
    for (int64_t i = 0; i < t->n_nodes; ++i) {
        const double v[3] = {x4[i].x, x4[i].y, x4[i].z};
        for (int k = 0; k < 3; ++k) {
            X[3 * i + k] = v[k];
            box_lo[k] = std::min(box_lo[k], v[k]);
            box_hi[k] = std::max(box_hi[k], v[k]);
        }
    }
    return FSI_OK;
}

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status fsi_mesh_create_tet(int64_t n_nodes, const double *X, int64_t n_tets,
                               const int32_t *tets, const fsi_physics *phys, int device,
                               void *cuda_stream, fsi_mesh **out)
{
    if (!out) return set_error(FSI_ERR_ARG, "out is NULL");
    *out = nullptr;
    fsi_tetmesh *t = nullptr;
    FSI_TRY(fsi_tetmesh_create(n_nodes, X, n_tets, tets, phys, device, cuda_stream, &t));
    fsi_mesh *m = new (std::nothrow) fsi_mesh();
    if (!m) {
        fsi_tetmesh_destroy(t);
        return set_error(FSI_ERR_OOM, "host allocation of the mesh handle failed");
    }
    m->phys = *phys;
    m->device = device;
    m->stream = (cudaStream_t)cuda_stream;
    m->n_nodes = n_nodes;
    m->n_elems = n_tets;
    m->alpha_m = t->alpha_m;
    m->alpha_f = t->alpha_f;
    m->gamma = t->gamma;
    m->tet = t;
    if (cudaMalloc(&m->dev_counters, 8 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        fsi_mesh_destroy(m);
        return set_error(FSI_ERR_OOM, "fsi_mesh_create_tet: cudaMalloc failed");
    }
    *out = m;
    return FSI_OK;
}


fsi_status fsi_tetmesh_create(int64_t n_nodes, const double *X, int64_t n_tets,
                              const int32_t *tets, const fsi_physics *phys, int device,
                              void *cuda_stream, fsi_tetmesh **out)
{
    if (!out) return set_error(FSI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_nodes < 4 || n_nodes >= INT32_MAX || n_tets < 1 || n_tets >= INT32_MAX / 4)
        return set_error(FSI_ERR_ARG, "fsi_tetmesh_create: bad sizes");
    if (!X || !tets || !phys) return set_error(FSI_ERR_ARG, "fsi_tetmesh_create: NULL argument");
    if (!(phys->rho > 0.0) || !(phys->mu >= 0.0) || !(phys->dt > 0.0) || !(phys->C_I >= 0.0) ||
        !(phys->C_T >= 0.0) || !(phys->rho_inf >= 0.0 && phys->rho_inf <= 1.0))
        return set_error(FSI_ERR_ARG, "invalid physics");
    FSI_DEVICE(device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // host copies for the set-up structures
    std::vector<int32_t> ht((size_t)n_tets * 4);
    std::vector<double> hx((size_t)n_nodes * 3);
    FSI_CUDA(cudaMemcpyAsync(ht.data(), tets, ht.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                             s), "copy tets");
    FSI_CUDA(cudaMemcpyAsync(hx.data(), X, hx.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy coordinates");
    FSI_CUDA(cudaStreamSynchronize(s), "sync");
    for (int32_t v : ht)
        if (v < 0 || v >= n_nodes) return set_error(FSI_ERR_ARG, "tet node index out of range");
    // node -> slots, increasing slot order
    std::vector<int32_t> nstart((size_t)n_nodes + 1, 0), nslot(ht.size());
    for (int32_t v : ht) nstart[(size_t)v + 1] += 1;
    for (int64_t i = 0; i < n_nodes; ++i) nstart[i + 1] += nstart[i];
    {
        std::vector<int32_t> cur(nstart.begin(), nstart.end() - 1);
        for (size_t sl = 0; sl < ht.size(); ++sl) nslot[cur[ht[sl]]++] = (int32_t)sl;
    }
    // greedy distance-2 colouring in node order: a node takes the smallest
    // colour no node of its elements holds yet
    std::vector<int32_t> hcol((size_t)n_nodes, -1);
    int ncol = 0;
    {
        std::vector<int64_t> seen;  // per colour: last node that saw it
        for (int64_t v = 0; v < n_nodes; ++v) {
            for (int k = nstart[v]; k < nstart[v + 1]; ++k) {
                const int64_t e = nslot[k] >> 2;
                for (int a = 0; a < 4; ++a) {
                    const int c = hcol[ht[4 * e + a]];
                    if (c >= 0) {
                        if ((size_t)c >= seen.size()) seen.resize(c + 1, -1);
                        seen[c] = v;
                    }
                }
            }
            int c = 0;
            while ((size_t)c < seen.size() && seen[c] == v) ++c;
            hcol[v] = c;
            ncol = std::max(ncol, c + 1);
        }
    }
    // bucket grid: about two elements per bucket, cells as cubic as the box allows
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = INFINITY;
        hi[k] = -INFINITY;
    }
    for (int64_t i = 0; i < n_nodes; ++i)
        for (int k = 0; k < 3; ++k) {
            const double v = hx[3 * i + k];
            if (!std::isfinite(v)) return set_error(FSI_ERR_ARG, "non-finite node coordinate");
            lo[k] = std::min(lo[k], v);
            hi[k] = std::max(hi[k], v);
        }
    double ext[3], vol = 1.0;
    for (int k = 0; k < 3; ++k) {
        ext[k] = std::max(hi[k] - lo[k], 1e-300);
        vol *= ext[k];
    }
    const double cell = std::cbrt(vol / std::max(1.0, n_tets / 2.0));
    int nb[3];
    for (int k = 0; k < 3; ++k)
        nb[k] = (int)std::min<double>(1024.0, std::max(1.0, std::ceil(ext[k] / cell)));
    double inv_cell[3];
    for (int k = 0; k < 3; ++k) inv_cell[k] = nb[k] / ext[k];
    const int64_t nbk = (int64_t)nb[0] * nb[1] * nb[2];
    std::vector<int32_t> bstart((size_t)nbk + 1, 0);
    std::vector<int> brange((size_t)n_tets * 6);
    for (int64_t e = 0; e < n_tets; ++e) {
        for (int k = 0; k < 3; ++k) {
            double mn = INFINITY, mx = -INFINITY;
            for (int a = 0; a < 4; ++a) {
                const double v = hx[3 * (size_t)ht[4 * e + a] + k];
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            const double pad = 1e-9 * ext[k];
            int i0 = (int)std::floor((mn - pad - lo[k]) * inv_cell[k]);
            int i1 = (int)std::floor((mx + pad - lo[k]) * inv_cell[k]);
            brange[6 * e + 2 * k] = std::max(0, std::min(nb[k] - 1, i0));
            brange[6 * e + 2 * k + 1] = std::max(0, std::min(nb[k] - 1, i1));
        }
        for (int z = brange[6 * e + 4]; z <= brange[6 * e + 5]; ++z)
            for (int y = brange[6 * e + 2]; y <= brange[6 * e + 3]; ++y)
                for (int x = brange[6 * e]; x <= brange[6 * e + 1]; ++x)
                    bstart[(size_t)(x + (int64_t)nb[0] * (y + (int64_t)nb[1] * z)) + 1] += 1;
    }
    for (int64_t b = 0; b < nbk; ++b) bstart[b + 1] += bstart[b];
    if ((int64_t)bstart[nbk] >= INT32_MAX) return set_error(FSI_ERR_ARG, "bucket lists too long");
    std::vector<int32_t> btets(bstart[nbk]);
    {
        std::vector<int32_t> cur(bstart.begin(), bstart.end() - 1);
        for (int64_t e = 0; e < n_tets; ++e)
            for (int z = brange[6 * e + 4]; z <= brange[6 * e + 5]; ++z)
                for (int y = brange[6 * e + 2]; y <= brange[6 * e + 3]; ++y)
                    for (int x = brange[6 * e]; x <= brange[6 * e + 1]; ++x)
                        btets[cur[x + (int64_t)nb[0] * (y + (int64_t)nb[1] * z)]++] = (int32_t)e;
    }

    fsi_tetmesh *m = new fsi_tetmesh();
    m->device = device;
    m->stream = s;
    m->n_nodes = n_nodes;
    m->n_elems = n_tets;
    m->phys = *phys;
    const double r = phys->rho_inf;
    m->alpha_m = 0.5 * (3.0 - r) / (1.0 + r);
    m->alpha_f = 1.0 / (1.0 + r);
    m->gamma = 0.5 + m->alpha_m - m->alpha_f;
    for (int k = 0; k < 3; ++k) {
        m->nb[k] = nb[k];
        m->lo[k] = lo[k];
        m->inv_cell[k] = inv_cell[k];
        m->box_lo[k] = lo[k] - 1e-9 * ext[k];
        m->box_hi[k] = hi[k] + 1e-9 * ext[k];
    }
    const int64_t ntmp = cell_table_scan_ints(n_tets) + 16;
    bool ok = cudaMalloc(&m->X64, n_nodes * sizeof(double4)) == cudaSuccess &&
              cudaMalloc(&m->X32, n_nodes * sizeof(float4)) == cudaSuccess &&
              cudaMalloc(&m->tets, n_tets * sizeof(int4)) == cudaSuccess &&
              cudaMalloc(&m->node_start, nstart.size() * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&m->node_slot, nslot.size() * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&m->bucket_start, bstart.size() * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&m->bucket_tets, std::max<size_t>(1, btets.size()) * sizeof(int32_t)) ==
                  cudaSuccess &&
              cudaMalloc(&m->slot_scratch, (size_t)n_tets * 4 * 32) == cudaSuccess &&
              cudaMalloc(&m->corner_scratch, (size_t)n_tets * 12 * 8) == cudaSuccess &&
              cudaMalloc(&m->fill, (size_t)(n_tets + 1) * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&m->scan_tmp, (size_t)ntmp * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&m->nout, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&m->colors, (size_t)n_nodes * sizeof(int32_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fsi_tetmesh_destroy(m);
        return set_error(FSI_ERR_OOM, "fsi_tetmesh_create: cudaMalloc failed");
    }
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    ok = cudaMemcpyAsync(m->tets, tets, n_tets * sizeof(int4), cudaMemcpyDeviceToDevice, s) ==
             cudaSuccess &&
         cudaMemsetAsync(m->scan_tmp, 0, (size_t)ntmp * sizeof(int32_t), s) == cudaSuccess &&
         up(m->node_start, nstart.data(), nstart.size() * sizeof(int32_t)) &&
         up(m->node_slot, nslot.data(), nslot.size() * sizeof(int32_t)) &&
         up(m->bucket_start, bstart.data(), bstart.size() * sizeof(int32_t)) &&
         (btets.empty() || up(m->bucket_tets, btets.data(), btets.size() * sizeof(int32_t))) &&
         up(m->colors, hcol.data(), hcol.size() * sizeof(int32_t));
    m->n_colors = ncol;
    if (!ok) {
        fsi_tetmesh_destroy(m);
        return set_error(FSI_ERR_CUDA, "fsi_tetmesh_create: copy failed");
    }
    pad_tet_coords_kernel<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, X, m->X64, m->X32);
    fsi_status st = check_launch("pad coordinates kernel");
    if (st == FSI_OK) st = check_cuda(cudaStreamSynchronize(s), "sync");
    if (st != FSI_OK) {
        fsi_tetmesh_destroy(m);
        return st;
    }
    *out = m;
    return FSI_OK;
}

void fsi_tetmesh_destroy(fsi_tetmesh *m)
{
    if (!m) return;
    fsi::DeviceGuard _fsi_device_guard(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->X64);
    cudaFree(m->X32);
    cudaFree(m->tets);
    cudaFree(m->node_start);
    cudaFree(m->node_slot);
    cudaFree(m->bucket_start);
    cudaFree(m->bucket_tets);
    cudaFree(m->slot_scratch);
    cudaFree(m->corner_scratch);
    cudaFree(m->fill);
    cudaFree(m->scan_tmp);
    cudaFree(m->nout);
    cudaFree(m->colors);
    for (void *g : m->geo) cudaFree(g);
    delete m;
}

fsi_status fsi_tet_residual(fsi_tetmesh *m, fsi_prec prec, const void *U, const void *A,
                            const void *f, void *R)
{
    FSI_TRY(validate_tetmesh(m));
    if (!U || !A || !R) return set_error(FSI_ERR_ARG, "fsi_tet_residual: NULL argument");
    FSI_DEVICE(m->device);
    if (prec == FSI_F64) return tet_vms<double, false>(m, U, A, f, nullptr, R);
    if (prec == FSI_DF64) return tet_vms<df64, false>(m, U, A, f, nullptr, R);
    if (prec == FSI_F32) return tet_vms<float, false>(m, U, A, f, nullptr, R);
    return set_error(FSI_ERR_ARG, "bad precision");
}

fsi_status fsi_tet_jacobian_apply(fsi_tetmesh *m, fsi_prec prec, const void *U, const void *A,
                                  const void *f, const void *x, void *Jx)
{
    FSI_TRY(validate_tetmesh(m));
    if (!U || !A || !x || !Jx) return set_error(FSI_ERR_ARG, "fsi_tet_jacobian_apply: NULL argument");
    FSI_DEVICE(m->device);
    if (prec == FSI_F64) return tet_vms<double, true>(m, U, A, f, x, Jx);
    if (prec == FSI_DF64) return tet_vms<df64, true>(m, U, A, f, x, Jx);
    if (prec == FSI_F32) return tet_vms<float, true>(m, U, A, f, x, Jx);
    return set_error(FSI_ERR_ARG, "bad precision");
}

fsi_status fsi_tet_locate(fsi_tetmesh *m, int64_t np, const double *P, int32_t *elem,
                          double *lam, int32_t *cell_start, int32_t *perm, int64_t *n_outside)
{
    FSI_TRY(validate_tetmesh(m));
    if (np < 0 || np >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_tet_locate: bad m");
    if (np > 0 && (!P || !elem || !lam))
        return set_error(FSI_ERR_ARG, "fsi_tet_locate: NULL P, elem or lam");
    if (perm != nullptr && cell_start == nullptr)
        return set_error(FSI_ERR_ARG, "fsi_tet_locate: perm given without cell_start");
    if (cell_start != nullptr && perm == nullptr && np > 0)
        return set_error(FSI_ERR_ARG, "fsi_tet_locate: cell_start given without perm");
    FSI_DEVICE(m->device);
    cudaStream_t s = m->stream;
    const int64_t E = m->n_elems;
    const bool table = cell_start != nullptr;
    FSI_CUDA(cudaMemsetAsync(m->nout, 0, sizeof(unsigned long long), s), "memset");
    if (table) FSI_CUDA(cudaMemsetAsync(m->fill, 0, (E + 1) * sizeof(int32_t), s), "memset");
    if (np > 0) {
        BucketArgs B;
        for (int k = 0; k < 3; ++k) {
            B.nb[k] = m->nb[k];
            B.lo[k] = m->lo[k];
            B.inv_cell[k] = m->inv_cell[k];
            B.box_lo[k] = m->box_lo[k];
            B.box_hi[k] = m->box_hi[k];
        }
        tet_locate_kernel<<<grid_for(np, 128), 128, 0, s>>>(
            np, B, m->X64, m->X32, m->tets, m->bucket_start, m->bucket_tets, P, elem, lam,
            table ? m->fill : nullptr, m->nout);
        FSI_TRY(check_launch("tet locate kernel"));
    }
    if (table) FSI_TRY(build_cell_table(s, E, np, elem, m->fill, m->scan_tmp, cell_start, perm));
    if (n_outside) {
        unsigned long long h = 0;
        FSI_CUDA(cudaMemcpyAsync(&h, m->nout, sizeof h, cudaMemcpyDeviceToHost, s), "memcpy");
        FSI_CUDA(cudaStreamSynchronize(s), "stream sync");
        *n_outside = (int64_t)h;
    }
    return FSI_OK;
}

fsi_status fsi_tet_interp(fsi_tetmesh *m, fsi_prec prec, int64_t np, const int32_t *elem,
                          const void *lam, const void *U, void *u)
{
    FSI_TRY(validate_tetmesh(m));
    if (np < 0 || np >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_tet_interp: bad m");
    if (np == 0) return FSI_OK;
    if (!elem || !lam || !U || !u) return set_error(FSI_ERR_ARG, "fsi_tet_interp: NULL argument");
    FSI_DEVICE(m->device);
    const int g = grid_for(np, 256);
    if (prec == FSI_F64)
        tet_interp_kernel<double><<<g, 256, 0, m->stream>>>(np, m->n_elems, m->tets, elem,
                                                            (const double *)lam,
                                                            (const vec4<double> *)U, (double *)u);
    else if (prec == FSI_DF64)
        tet_interp_kernel<df64><<<g, 256, 0, m->stream>>>(np, m->n_elems, m->tets, elem,
                                                          (const double *)lam,
                                                          (const vec4<double> *)U, (double *)u);
    else if (prec == FSI_F32)
        tet_interp_kernel<float><<<g, 256, 0, m->stream>>>(np, m->n_elems, m->tets, elem,
                                                           (const float *)lam,
                                                           (const vec4<float> *)U, (float *)u);
    else
        return set_error(FSI_ERR_ARG, "bad precision");
    return check_launch("tet interp kernel");
}

fsi_status fsi_tet_spread(fsi_tetmesh *m, fsi_prec prec, int64_t np, const int32_t *elem,
                          const void *lam, const int32_t *cell_start, const int32_t *perm,
                          const void *lamv, const void *w, void *F, int accumulate)
{
    (void)elem;
    FSI_TRY(validate_tetmesh(m));
    if (np < 0 || np >= INT32_MAX) return set_error(FSI_ERR_ARG, "fsi_tet_spread: bad m");
    if (!F || !cell_start) return set_error(FSI_ERR_ARG, "fsi_tet_spread: NULL F or cell_start");
    if (np > 0 && (!lam || !perm || !lamv))
        return set_error(FSI_ERR_ARG, "fsi_tet_spread: NULL lam, perm or forces");
    FSI_DEVICE(m->device);
    const int64_t E = m->n_elems;
    const int cg = grid_for((E + 7) / 8 * 32, 256, sm_count() * 64);
    const int ng = grid_for(m->n_nodes, 256);
    cudaStream_t s = m->stream;
    if (prec == FSI_F64) {
        tet_spread_cells_kernel<double><<<cg, 256, 0, s>>>(E, (const double *)lam, cell_start, perm,
                                                           (const double *)lamv,
                                                           (const double *)w,
                                                           (double *)m->corner_scratch);
        FSI_TRY(check_launch("tet spread cells kernel"));
        tet_spread_nodes_kernel<double><<<ng, 256, 0, s>>>(m->n_nodes, m->node_start, m->node_slot,
                                                           cell_start,
                                                           (const double *)m->corner_scratch,
                                                           (double *)F, accumulate);
    } else if (prec == FSI_DF64) {
        tet_spread_cells_kernel<df64><<<cg, 256, 0, s>>>(E, (const double *)lam, cell_start, perm,
                                                         (const double *)lamv, (const double *)w,
                                                         (df64 *)m->corner_scratch);
        FSI_TRY(check_launch("tet spread cells kernel"));
        tet_spread_nodes_kernel<df64><<<ng, 256, 0, s>>>(m->n_nodes, m->node_start, m->node_slot,
                                                         cell_start,
                                                         (const df64 *)m->corner_scratch,
                                                         (double *)F, accumulate);
    } else if (prec == FSI_F32) {
        tet_spread_cells_kernel<float><<<cg, 256, 0, s>>>(E, (const float *)lam, cell_start, perm,
                                                          (const float *)lamv, (const float *)w,
                                                          (float *)m->corner_scratch);
        FSI_TRY(check_launch("tet spread cells kernel"));
        tet_spread_nodes_kernel<float><<<ng, 256, 0, s>>>(m->n_nodes, m->node_start, m->node_slot,
                                                          cell_start,
                                                          (const float *)m->corner_scratch,
                                                          (float *)F, accumulate);
    } else {
        return set_error(FSI_ERR_ARG, "bad precision");
    }
    return check_launch("tet spread nodes kernel");
}

}  // extern "C"
