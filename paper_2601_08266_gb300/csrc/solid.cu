// solid.cu -- the immersed hyperelastic solid of Sec. 2.2 on a Q1 hexahedral
// solid mesh (Eq. solid_weak_form):
//
//   R^s_a = sum_g N_a (rho_s - rho_f)(uddot(g) - f) detJ0            (inertia)
//         + sum_g P(F) grad_X N_a detJ0                              (int grad w : sigma)
//         - sum_g 2 mu_f D grad_x N_a J detJ0                        (artificial fluid)
//
// with the compressible neo-Hookean P = mu (F - F^-T) + lam ln J F^-T, 2x2x2
// Gauss points in the reference configuration, D the symmetric velocity
// gradient of the solid's own velocity field on the configuration at the
// start of the step (frozen like C), and generalized-alpha / Newmark
// kinematics: the residual is taken at uddot_{n+alpha_m}, v_{n+alpha_f},
// u_{n+alpha_f}, all functions of uddot_{n+1} = C^T Vdot_{n+1} (the solid
// nodes are the Lagrange multiplier points, Sec. 2.3).  The linearisation
// w.r.t. uddot_{n+1} carries the chain factors alpha_m (inertia),
// alpha_f beta dt^2 (stress), alpha_f gamma dt (viscous).
//
// GPU layout: one thread per element computes its 8 x 3 nodal contributions
// (geometry from the reference coordinates at each Gauss point) into an
// element scratch [es][8][3]; each node then sums its element slots through a
// node -> (element, corner) table in a fixed order.  No atomics;
// deterministic.
#include <cmath>
#include <vector>

#include "fsi_internal.cuh"

struct fsi_solid {
    fsi_mesh *mesh;
    int64_t ns, es;
    double *X;           // [ns][3] reference coordinates
    int32_t *conn;       // [es][8]
    int32_t *node_start; // [ns+1] CSR of element slots e*8+a per node
    int32_t *node_slot;  // [es*8]
    void *elem_f;        // [es][8][3] scratch, 8 bytes per value
    double rho_s, mu_s, lam_s;
};

namespace fsi {
namespace {

template <typename T> struct M3 {
    T a[3][3];
};

template <typename T> __device__ __forceinline__ T det3(const M3<T> &m)
{
    return m.a[0][0] * (m.a[1][1] * m.a[2][2] - m.a[1][2] * m.a[2][1]) -
           m.a[0][1] * (m.a[1][0] * m.a[2][2] - m.a[1][2] * m.a[2][0]) +
           m.a[0][2] * (m.a[1][0] * m.a[2][1] - m.a[1][1] * m.a[2][0]);
}

// inverse by cofactors; returns the determinant
template <typename T> __device__ __forceinline__ T inv3(const M3<T> &m, M3<T> &r)
{
    const T d = det3(m);
    const T id = T(1) / d;
    r.a[0][0] = (m.a[1][1] * m.a[2][2] - m.a[1][2] * m.a[2][1]) * id;
    r.a[0][1] = (m.a[0][2] * m.a[2][1] - m.a[0][1] * m.a[2][2]) * id;
    r.a[0][2] = (m.a[0][1] * m.a[1][2] - m.a[0][2] * m.a[1][1]) * id;
    r.a[1][0] = (m.a[1][2] * m.a[2][0] - m.a[1][0] * m.a[2][2]) * id;
    r.a[1][1] = (m.a[0][0] * m.a[2][2] - m.a[0][2] * m.a[2][0]) * id;
    r.a[1][2] = (m.a[0][2] * m.a[1][0] - m.a[0][0] * m.a[1][2]) * id;
    r.a[2][0] = (m.a[1][0] * m.a[2][1] - m.a[1][1] * m.a[2][0]) * id;
    r.a[2][1] = (m.a[0][1] * m.a[2][0] - m.a[0][0] * m.a[2][1]) * id;
    r.a[2][2] = (m.a[0][0] * m.a[1][1] - m.a[0][1] * m.a[1][0]) * id;
    return d;
}

template <typename T> __device__ __forceinline__ T log_t(T v);
template <> __device__ __forceinline__ double log_t(double v) { return log(v); }
template <> __device__ __forceinline__ float log_t(float v) { return logf(v); }

struct SolidArgs {
    int64_t es;
    const double *X;
    const int32_t *conn;
    double drho, mu, lam, mu_f;
    double g[3];
    double c_a, c_u, c_v;  // tangent chain factors
};

// MODE 0: residual from (u_af, v_af, a_am, u_n); MODE 1: tangent apply along x
// at (u_af, u_n).  T is the arithmetic and the array type of u_af, v_af,
// a_am, x; u_n and X are FP64.
template <typename T, int MODE>
__global__ void solid_elem_kernel(SolidArgs s, const T *__restrict__ u_af, const T *__restrict__ v_af,
                                  const T *__restrict__ a_am, const double *__restrict__ u_n,
                                  const T *__restrict__ x, T *__restrict__ ef)
{
    const T gq = T(0.57735026918962576451);  // 1/sqrt(3)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.es;
         e += (int64_t)gridDim.x * blockDim.x) {
        int nd[8];
        T Xe[8][3], ue[8][3], un[8][3], ve[8][3], ae[8][3];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            nd[a] = s.conn[8 * e + a];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int64_t q = 3 * (int64_t)nd[a] + i;
                Xe[a][i] = (T)s.X[q];
                ue[a][i] = u_af[q];
                un[a][i] = (T)u_n[q];
                ve[a][i] = MODE == 0 ? v_af[q] : x[q];
                ae[a][i] = MODE == 0 ? a_am[q] : x[q];
            }
        }
        T out[8][3];
#pragma unroll
        for (int a = 0; a < 8; ++a) out[a][0] = out[a][1] = out[a][2] = T(0);
        for (int qp = 0; qp < 8; ++qp) {
            const T xi[3] = {(qp & 1) ? gq : -gq, (qp & 2) ? gq : -gq, (qp & 4) ? gq : -gq};
            T N[8], dN[8][3];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                T f[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) f[k] = T(0.5) * (T(1) + (((a >> k) & 1) ? xi[k] : -xi[k]));
                N[a] = f[0] * f[1] * f[2];
                dN[a][0] = T(0.5) * (((a >> 0) & 1) ? T(1) : T(-1)) * f[1] * f[2];
                dN[a][1] = T(0.5) * (((a >> 1) & 1) ? T(1) : T(-1)) * f[0] * f[2];
                dN[a][2] = T(0.5) * (((a >> 2) & 1) ? T(1) : T(-1)) * f[0] * f[1];
            }
            // reference geometry: J0[i][k] = sum_a X_ai dN_a/dxi_k
            M3<T> J0, J0i;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    T t = T(0);
#pragma unroll
                    for (int a = 0; a < 8; ++a) t += Xe[a][i] * dN[a][k];
                    J0.a[i][k] = t;
                }
            const T det0 = inv3(J0, J0i);
            T gX[8][3];  // grad_X N_a = J0^{-T} dN_a/dxi
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    gX[a][j] = dN[a][0] * J0i.a[0][j] + dN[a][1] * J0i.a[1][j] + dN[a][2] * J0i.a[2][j];
            // deformation gradient at the alpha level
            M3<T> F, Fi;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    T t = i == j ? T(1) : T(0);
#pragma unroll
                    for (int a = 0; a < 8; ++a) t += ue[a][i] * gX[a][j];
                    F.a[i][j] = t;
                }
            const T J = inv3(F, Fi);
            const T lnJ = log_t(J);
            const T mu = (T)s.mu, lam = (T)s.lam;
            M3<T> P;
            if (MODE == 0) {
                // P = mu (F - F^-T) + lam ln J F^-T
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        P.a[i][j] = mu * (F.a[i][j] - Fi.a[j][i]) + lam * lnJ * Fi.a[j][i];
            } else {
                // dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T,
                // dF = c_u sum_a x_a (x) grad_X N_a
                M3<T> dF;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        T t = T(0);
#pragma unroll
                        for (int a = 0; a < 8; ++a) t += ae[a][i] * gX[a][j];
                        dF.a[i][j] = (T)s.c_u * t;
                    }
                T tr = T(0);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) tr += Fi.a[i][k] * dF.a[k][i];
                // B = F^-T dF^T F^-T: B_ij = sum_kl Fi_ki dF_lk Fi_jl
                M3<T> B1;  // dF^T F^-T: (B1)_kj = sum_l dF_lk Fi_jl
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        B1.a[k][j] = dF.a[0][k] * Fi.a[j][0] + dF.a[1][k] * Fi.a[j][1] + dF.a[2][k] * Fi.a[j][2];
                const T c1 = mu - lam * lnJ, c2 = lam * tr;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const T Bij = Fi.a[0][i] * B1.a[0][j] + Fi.a[1][i] * B1.a[1][j] + Fi.a[2][i] * B1.a[2][j];
                        P.a[i][j] = mu * dF.a[i][j] + c1 * Bij + c2 * Fi.a[j][i];
                    }
            }
            // inertia: N_a drho (uddot(g) - f) (MODE 1: c_a drho N_a x(g))
            T ag[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T t = T(0);
#pragma unroll
                for (int a = 0; a < 8; ++a) t += N[a] * ae[a][i];
                ag[i] = MODE == 0 ? (T)s.drho * (t - (T)s.g[i]) : (T)(s.c_a * s.drho) * t;
            }
            // viscous: configuration at the start of the step
            M3<T> Fn, Fni;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    T t = i == j ? T(1) : T(0);
#pragma unroll
                    for (int a = 0; a < 8; ++a) t += un[a][i] * gX[a][j];
                    Fn.a[i][j] = t;
                }
            const T Jn = inv3(Fn, Fni);
            T gx[8][3];  // grad_x N_a = grad_X N_a F_n^{-1}
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    gx[a][j] = gX[a][0] * Fni.a[0][j] + gX[a][1] * Fni.a[1][j] + gX[a][2] * Fni.a[2][j];
            M3<T> L;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    T t = T(0);
#pragma unroll
                    for (int a = 0; a < 8; ++a) t += ve[a][i] * gx[a][j];
                    L.a[i][j] = t;
                }
            const T vs = (T)(2.0 * s.mu_f) * Jn * (MODE == 0 ? T(1) : (T)s.c_v);
            M3<T> D;  // 2 mu_f J_n D (times c_v for the tangent)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) D.a[i][j] = vs * T(0.5) * (L.a[i][j] + L.a[j][i]);
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T fint = P.a[i][0] * gX[a][0] + P.a[i][1] * gX[a][1] + P.a[i][2] * gX[a][2];
                    const T fvis = D.a[i][0] * gx[a][0] + D.a[i][1] * gx[a][1] + D.a[i][2] * gx[a][2];
                    out[a][i] += det0 * (N[a] * ag[i] + fint - fvis);
                }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) ef[(8 * e + a) * 3 + i] = out[a][i];
    }
}

// R_b = sum of the element slots of node b (fixed order), overwrite
template <typename T>
__global__ void solid_gather_kernel(int64_t ns, const int32_t *__restrict__ start,
                                    const int32_t *__restrict__ slot, const T *__restrict__ ef,
                                    T *__restrict__ R)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < ns;
         b += (int64_t)gridDim.x * blockDim.x) {
        T r0 = T(0), r1 = T(0), r2 = T(0);
        for (int q = start[b]; q < start[b + 1]; ++q) {
            const T *p = ef + 3 * (int64_t)slot[q];
            r0 += p[0];
            r1 += p[1];
            r2 += p[2];
        }
        R[3 * b] = r0;
        R[3 * b + 1] = r1;
        R[3 * b + 2] = r2;
    }
}

// generalized-alpha / Newmark stage values from uddot_{n+1}
__global__ void solid_stage_kernel(int64_t n3, double dt, double am, double af, double gm,
                                   double beta, const double *u, const double *v, const double *a,
                                   const double *a1, double *u_af, double *v_af, double *a_am)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double v1 = v[q] + dt * ((1.0 - gm) * a[q] + gm * a1[q]);
        const double u1 = u[q] + dt * v[q] + dt * dt * ((0.5 - beta) * a[q] + beta * a1[q]);
        u_af[q] = u[q] + af * (u1 - u[q]);
        v_af[q] = v[q] + af * (v1 - v[q]);
        a_am[q] = a[q] + am * (a1[q] - a[q]);
    }
}

// history advance: (u, v, a) <- (u_{n+1}, v_{n+1}, uddot_{n+1})
__global__ void solid_advance_kernel(int64_t n3, double dt, double gm, double beta, double *u,
                                     double *v, double *a, const double *a1)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double v1 = v[q] + dt * ((1.0 - gm) * a[q] + gm * a1[q]);
        const double u1 = u[q] + dt * v[q] + dt * dt * ((0.5 - beta) * a[q] + beta * a1[q]);
        u[q] = u1;
        v[q] = v1;
        a[q] = a1[q];
    }
}

__global__ void positions_kernel(int64_t n3, const double *X, const double *u, double *x)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
         q += (int64_t)gridDim.x * blockDim.x)
        x[q] = X[q] + u[q];
}

int grid_of(int64_t n, int threads = 128)
{
    const int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > sm_count() * 32 ? sm_count() * 32 : b));
}

SolidArgs args_of(const fsi_solid *b, const double g[3])
{
    const fsi_mesh *m = b->mesh;
    SolidArgs s;
    s.es = b->es;
    s.X = b->X;
    s.conn = b->conn;
    s.drho = b->rho_s - m->phys.rho;
    s.mu = b->mu_s;
    s.lam = b->lam_s;
    s.mu_f = m->phys.mu;
    for (int i = 0; i < 3; ++i) s.g[i] = g ? g[i] : 0.0;
    const double beta = 0.25 * (1.0 + m->alpha_m - m->alpha_f) * (1.0 + m->alpha_m - m->alpha_f);
    const double dt = m->phys.dt;
    s.c_a = m->alpha_m;
    s.c_u = m->alpha_f * beta * dt * dt;
    s.c_v = m->alpha_f * m->gamma * dt;
    return s;
}

}  // namespace

// ---------------------------------------------------------------- internal API
fsi_status solid_residual_impl(fsi_solid *b, const double *u_af, const double *v_af,
                               const double *a_am, const double *u_n, const double g[3], double *R)
{
    cudaStream_t s = b->mesh->stream;
    solid_elem_kernel<double, 0><<<grid_of(b->es), 128, 0, s>>>(
        args_of(b, g), u_af, v_af, a_am, u_n, nullptr, (double *)b->elem_f);
    FSI_TRY(check_launch("solid element kernel"));
    solid_gather_kernel<double><<<grid_of(b->ns, 256), 256, 0, s>>>(
        b->ns, b->node_start, b->node_slot, (const double *)b->elem_f, R);
    return check_launch("solid gather kernel");
}

template <typename T>
fsi_status solid_tangent_impl(fsi_solid *b, const T *u_af, const double *u_n, const T *x, T *Jx)
{
    cudaStream_t s = b->mesh->stream;
    solid_elem_kernel<T, 1><<<grid_of(b->es), 128, 0, s>>>(args_of(b, nullptr), u_af, nullptr,
                                                          nullptr, u_n, x, (T *)b->elem_f);
    FSI_TRY(check_launch("solid element kernel"));
    solid_gather_kernel<T><<<grid_of(b->ns, 256), 256, 0, s>>>(
        b->ns, b->node_start, b->node_slot, (const T *)b->elem_f, Jx);
    return check_launch("solid gather kernel");
}
template fsi_status solid_tangent_impl<double>(fsi_solid *, const double *, const double *,
                                               const double *, double *);
template fsi_status solid_tangent_impl<float>(fsi_solid *, const float *, const double *,
                                              const float *, float *);

fsi_status solid_stage_impl(fsi_solid *b, const double *u, const double *v, const double *a,
                            const double *a1, double *u_af, double *v_af, double *a_am)
{
    const fsi_mesh *m = b->mesh;
    const double beta = 0.25 * (1.0 + m->alpha_m - m->alpha_f) * (1.0 + m->alpha_m - m->alpha_f);
    solid_stage_kernel<<<grid_of(3 * b->ns, 256), 256, 0, m->stream>>>(
        3 * b->ns, m->phys.dt, m->alpha_m, m->alpha_f, m->gamma, beta, u, v, a, a1, u_af, v_af,
        a_am);
    return check_launch("solid stage kernel");
}

int64_t solid_nodes(const fsi_solid *b) { return b->ns; }

}  // namespace fsi

// ---------------------------------------------------------------- C ABI
using namespace fsi;

extern "C" {

fsi_status fsi_solid_create(fsi_mesh *mesh, int64_t n_nodes, int64_t n_elems, const double *X,
                            const int32_t *conn, double rho_s, double mu_s, double lambda_s,
                            fsi_solid **out)
{
    FSI_TRY(validate_mesh(mesh));
    if (!out) return set_error(FSI_ERR_ARG, "fsi_solid_create: out is NULL");
    *out = nullptr;
    if (n_nodes < 1 || n_elems < 1 || n_nodes > INT32_MAX / 3 || n_elems > INT32_MAX / 8)
        return set_error(FSI_ERR_ARG, "fsi_solid_create: sizes out of range");
    if (!X || !conn) return set_error(FSI_ERR_ARG, "fsi_solid_create: NULL array");
    if (!(rho_s > 0.0) || !(mu_s > 0.0) || !(lambda_s >= 0.0))
        return set_error(FSI_ERR_ARG, "fsi_solid_create: rho_s, mu_s > 0 and lambda_s >= 0");
    FSI_DEVICE(mesh->device);
    // node -> element-slot table, built on the host from the connectivity
    std::vector<int32_t> hconn((size_t)n_elems * 8);
    FSI_CUDA(cudaMemcpy(hconn.data(), conn, hconn.size() * sizeof(int32_t), cudaMemcpyDeviceToHost),
             "memcpy");
    std::vector<int32_t> start((size_t)n_nodes + 1, 0), slot(hconn.size());
    for (int32_t v : hconn) {
        if (v < 0 || v >= n_nodes)
            return set_error(FSI_ERR_ARG, "fsi_solid_create: connectivity entry %d out of range", v);
        start[(size_t)v + 1]++;
    }
    for (int64_t b = 0; b < n_nodes; ++b) start[b + 1] += start[b];
    {
        std::vector<int32_t> fill(start.begin(), start.end() - 1);
        for (size_t q = 0; q < hconn.size(); ++q) slot[fill[hconn[q]]++] = (int32_t)q;
    }
    fsi_solid *b = new (std::nothrow) fsi_solid();
    if (!b) return set_error(FSI_ERR_OOM, "host allocation failed");
    b->mesh = mesh;
    b->ns = n_nodes;
    b->es = n_elems;
    b->rho_s = rho_s;
    b->mu_s = mu_s;
    b->lam_s = lambda_s;
    struct {
        void **p;
        size_t bytes;
    } req[] = {{(void **)&b->X, (size_t)n_nodes * 3 * sizeof(double)},
               {(void **)&b->conn, hconn.size() * sizeof(int32_t)},
               {(void **)&b->node_start, start.size() * sizeof(int32_t)},
               {(void **)&b->node_slot, slot.size() * sizeof(int32_t)},
               {&b->elem_f, (size_t)n_elems * 24 * sizeof(double)}};
    for (auto &r : req) {
        if (cudaMalloc(r.p, r.bytes) != cudaSuccess) {
            cudaGetLastError();
            fsi_solid_destroy(b);
            return set_error(FSI_ERR_OOM, "fsi_solid_create: cudaMalloc failed");
        }
    }
    cudaError_t e = cudaMemcpy(b->X, X, (size_t)n_nodes * 3 * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->conn, conn, hconn.size() * sizeof(int32_t), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->node_start, start.data(), start.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->node_slot, slot.data(), slot.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        fsi_solid_destroy(b);
        return check_cuda(e, "fsi_solid_create: copy");
    }
    *out = b;
    return FSI_OK;
}

void fsi_solid_destroy(fsi_solid *b)
{
    if (!b) return;
    fsi::DeviceGuard _fsi_device_guard(b->mesh->device);
    cudaStreamSynchronize(b->mesh->stream);
    cudaFree(b->X);
    cudaFree(b->conn);
    cudaFree(b->node_start);
    cudaFree(b->node_slot);
    cudaFree(b->elem_f);
    delete b;
}

fsi_status fsi_solid_residual(fsi_solid *b, const double *u_af, const double *v_af,
                              const double *a_am, const double *u_n, const double *g, double *R)
{
    if (!b) return set_error(FSI_ERR_ARG, "fsi_solid_residual: solid is NULL");
    if (!u_af || !v_af || !a_am || !u_n || !R)
        return set_error(FSI_ERR_ARG, "fsi_solid_residual: NULL argument");
    FSI_DEVICE(b->mesh->device);
    return solid_residual_impl(b, u_af, v_af, a_am, u_n, g, R);
}

fsi_status fsi_solid_tangent_apply(fsi_solid *b, fsi_prec prec, const void *u_af, const double *u_n,
                                   const void *x, void *Jx)
{
    if (!b) return set_error(FSI_ERR_ARG, "fsi_solid_tangent_apply: solid is NULL");
    if (!u_af || !u_n || !x || !Jx)
        return set_error(FSI_ERR_ARG, "fsi_solid_tangent_apply: NULL argument");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(b->mesh->device);
    if (prec == FSI_F64)
        return solid_tangent_impl<double>(b, (const double *)u_af, u_n, (const double *)x,
                                          (double *)Jx);
    return solid_tangent_impl<float>(b, (const float *)u_af, u_n, (const float *)x, (float *)Jx);
}

fsi_status fsi_solid_stage(fsi_solid *b, const double *u, const double *v, const double *a,
                           const double *a_next, double *u_af, double *v_af, double *a_am)
{
    if (!b || !u || !v || !a || !a_next || !u_af || !v_af || !a_am)
        return set_error(FSI_ERR_ARG, "fsi_solid_stage: NULL argument");
    FSI_DEVICE(b->mesh->device);
    return solid_stage_impl(b, u, v, a, a_next, u_af, v_af, a_am);
}

fsi_status fsi_solid_advance(fsi_solid *b, double *u, double *v, double *a, const double *a_next)
{
    if (!b || !u || !v || !a || !a_next)
        return set_error(FSI_ERR_ARG, "fsi_solid_advance: NULL argument");
    FSI_DEVICE(b->mesh->device);
    const fsi_mesh *m = b->mesh;
    const double beta = 0.25 * (1.0 + m->alpha_m - m->alpha_f) * (1.0 + m->alpha_m - m->alpha_f);
    solid_advance_kernel<<<grid_of(3 * b->ns, 256), 256, 0, m->stream>>>(
        3 * b->ns, m->phys.dt, m->gamma, beta, u, v, a, a_next);
    return check_launch("solid advance kernel");
}

fsi_status fsi_solid_positions(fsi_solid *b, const double *u, double *x)
{
    if (!b || !u || !x) return set_error(FSI_ERR_ARG, "fsi_solid_positions: NULL argument");
    FSI_DEVICE(b->mesh->device);
    positions_kernel<<<grid_of(3 * b->ns, 256), 256, 0, b->mesh->stream>>>(3 * b->ns, b->X, u, x);
    return check_launch("solid positions kernel");
}

}  // extern "C"
