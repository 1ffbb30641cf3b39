// newton.cu -- the implicit step on the reduced FSI system (Sec. 2.4 of the
// paper): coupled residual and Jacobian (fluid VMS operators plus the solid
// coupling C W D C^T through interpolation and spreading), a nodal 4x4
// block-Jacobi preconditioner built by colour probing, restarted GMRES with
// classical Gram-Schmidt and one reorthogonalisation (FP64 dot products), and
// Newton with an FP64 residual and update.  In mixed mode the Krylov vectors,
// Jacobian applies and preconditioner run in FP32 (defect correction).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "df64.cuh"
#include "fsi_internal.cuh"

namespace fsi {
namespace {

constexpr int kRedGrid = 456;   // fixed partial-sum grid (3 CTAs per SM): deterministic dots
// fixed grid of the multi-update pass (4 CTAs per SM: its |w|^2 partials,
// one row of kAxpyGrid; the multi-dot's 76 registers keep it at 3)
constexpr int kAxpyGrid = 608;
constexpr int kRedThreads = 256;
constexpr int kDotGroup = 8;    // vectors per multi-dot pass
static_assert(kDotGroup % 2 == 0, "the FP32 multi-dot pairs vectors");

int grid1d(int64_t n, int threads = 256, int cap = sm_count() * 16)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

#define GRID_STRIDE(i, n)                                                                  \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n);              \
         i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------ elementwise
template <typename Ti, typename To> __global__ void cast_kernel(int64_t n, const Ti *a, To *b)
{
    GRID_STRIDE(i, n) b[i] = (To)a[i];
}

template <typename T> __global__ void neg_cast_kernel(int64_t n, const double *a, T *b)
{
    GRID_STRIDE(i, n) b[i] = (T)(-a[i]);
}

template <typename T> __global__ void add_to_f64_kernel(int64_t n, const T *x, double *y)
{
    GRID_STRIDE(i, n) y[i] += (double)x[i];
}

template <typename T> __global__ void zero_kernel(int64_t n, T *x)
{
    GRID_STRIDE(i, n) x[i] = T(0);
}

template <typename T> __global__ void add_kernel(int64_t n, const T *x, T *y)
{
    GRID_STRIDE(i, n) y[i] += x[i];
}

template <typename T> __global__ void sub_kernel(int64_t n, const T *a, const T *b, T *c)
{
    GRID_STRIDE(i, n) c[i] = a[i] - b[i];
}

// V_{n+1} = V_n + dt Vdot_n + gamma dt (Vdot_{n+1} - Vdot_n), slot 4 = 0
__global__ void velocity_next_kernel(int64_t n, double dt, double gamma, const double *y,
                                     const double *Vn, const double *An, double *V1)
{
    GRID_STRIDE(i, n)
    {
        for (int c = 0; c < 3; ++c) {
            const int64_t k = 4 * i + c;
            V1[k] = Vn[k] + dt * An[k] + gamma * dt * (y[k] - An[k]);
        }
        V1[4 * i + 3] = 0.0;
    }
}

// r^s_B = drho (a_B - g) + k dt (C^T V_{n+1})_B for inside points, 0 outside
__global__ void solid_force_kernel(int64_t m, const int32_t *elem, const double *a,
                                   const double *v1, double drho, double kdt, double g0,
                                   double g1, double g2, double *rs)
{
    GRID_STRIDE(b, m)
    {
        const bool in = elem[b] >= 0;
        const double g[3] = {g0, g1, g2};
        for (int c = 0; c < 3; ++c)
            rs[3 * b + c] = in ? drho * (a[3 * b + c] - g[c]) + kdt * v1[3 * b + c] : 0.0;
    }
}

// y[i].xyz += f[i].xyz (the coupling's nodal forces into the Jacobian apply)
template <typename T>
__global__ void add_xyz_kernel(int64_t n, const vec4<T> *__restrict__ f, vec4<T> *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const vec4<T> a = f[i];
        vec4<T> b = y[i];
        b.x += a.x;
        b.y += a.y;
        b.z += a.z;
        y[i] = b;
    }
}

// the same followed by the Dirichlet rows (Jx = x where mask), one pass
template <typename T>
__global__ void add_xyz_rows_kernel(int64_t n, const vec4<T> *__restrict__ f,
                                    const uchar4 *__restrict__ mask, const vec4<T> *__restrict__ x,
                                    vec4<T> *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const vec4<T> a = f[i];
        const uchar4 mk = mask[i];
        vec4<T> b = y[i];
        b.x += a.x;
        b.y += a.y;
        b.z += a.z;
        if (mk.x | mk.y | mk.z | mk.w) {
            const vec4<T> xv = x[i];
            if (mk.x) b.x = xv.x;
            if (mk.y) b.y = xv.y;
            if (mk.z) b.z = xv.z;
            if (mk.w) b.w = xv.w;
        }
        y[i] = b;
    }
}

template <typename T> __global__ void scale_kernel(int64_t n, T alpha, const T *x, T *y)
{
    GRID_STRIDE(i, n) y[i] = alpha * x[i];
}

__global__ void dirichlet_residual_kernel(int64_t n4, const uint8_t *mask, const double *y,
                                          const double *yD, double *R)
{
    GRID_STRIDE(i, n4)
    if (mask[i]) R[i] = y[i] - yD[i];
}

template <typename T>
__global__ void dirichlet_rows_kernel(int64_t n4, const uint8_t *mask, const T *x, T *Jx)
{
    GRID_STRIDE(i, n4)
    if (mask[i]) Jx[i] = x[i];
}

// ------------------------------------------------------------ reductions
// partial[k][block] = sum over the block's grid-stride range of V_k . w, for
// k in [k0, k0+cnt); fixed grid and block size (deterministic).  FP64 vectors
// accumulate in FP64.  FP32 vectors accumulate FP64-grade on the FP32 pipe
// (GB300's FP64 unit is ~70x slower): each product is exact as the pair
// (p, e) of an FMA-based TwoProd; p joins the running float sum s by Knuth's
// TwoSum, whose rounding error t and e go to a float compensation c, and
// (s, c) is renormalised (Fast2Sum) once per 4-value record: 10 FP32
// instructions per product against 13 for a full double-float addition, with
// |c| kept below a few ulp(s) so the error stays at the double-float level.
struct Comp {
    float s, c;
    __device__ Comp() {}
    __device__ explicit Comp(int) : s(0.0f), c(0.0f) {}
};
__device__ __forceinline__ void dot_acc(double &acc, double v, double w) { acc += v * w; }
__device__ __forceinline__ void dot_acc(Comp &acc, float v, float w)
{
    const float p = __fmul_rn(v, w);
    const float e = __fmaf_rn(v, w, -p);
    const float s = __fadd_rn(acc.s, p);
    const float bb = __fsub_rn(s, acc.s);
    const float t = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.s = s;
    acc.c = __fadd_rn(acc.c, __fadd_rn(e, t));
}
// the same for two accumulators at once on the paired FP32 instructions
// (FMUL2, FFMA2, FADD2): each half rounds exactly like the scalar
// operation, so the two sums equal two scalar Comp sums bit for bit, at half
// the issue slots
struct Comp2 {
    float2 s, c;
};
__device__ __forceinline__ float2 negf2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void dot_acc2(Comp2 &acc, float2 v, float2 w)
{
    const float2 p = __fmul2_rn(v, w);
    const float2 e = __ffma2_rn(v, w, negf2(p));
    const float2 s = __fadd2_rn(acc.s, p);
    const float2 bb = __fadd2_rn(s, negf2(acc.s));
    const float2 t = __fadd2_rn(__fadd2_rn(acc.s, negf2(__fadd2_rn(s, negf2(bb)))),
                                __fadd2_rn(p, negf2(bb)));
    acc.s = s;
    acc.c = __fadd2_rn(acc.c, __fadd2_rn(e, t));
}
__device__ __forceinline__ void dot_renorm2(Comp2 &acc)
{
    const float2 s = __fadd2_rn(acc.s, acc.c);
    acc.c = __fadd2_rn(acc.c, negf2(__fadd2_rn(s, negf2(acc.s))));
    acc.s = s;
}
__device__ __forceinline__ void dot_renorm(double &) {}
__device__ __forceinline__ void dot_renorm(Comp &acc)
{
    const float s = __fadd_rn(acc.s, acc.c);
    acc.c = __fsub_rn(acc.c, __fsub_rn(s, acc.s));
    acc.s = s;
}
__device__ __forceinline__ double dot_value(double a) { return a; }
__device__ __forceinline__ double dot_value(Comp a) { return (double)a.s + (double)a.c; }
template <typename T> struct DotAcc {
    using type = double;
};
template <> struct DotAcc<float> {
    using type = Comp;
};

// (index self_k, when in [k0, k0+cnt), stands for w itself: w . w)
// (cond, when not null, is a device flag: the kernel does nothing when it is 0)
template <typename T>
__global__ void __launch_bounds__(kRedThreads, 3) multi_dot_partial_kernel(
    int k0, int cnt, int64_t len4, const vec4<T> *V, int64_t vstride, const vec4<T> *w,
    double *partial, int self_k, const double *cond)
{
    if (cond && *cond == 0.0) return;
    using Acc = typename DotAcc<T>::type;
    __shared__ double red[kDotGroup][kRedThreads / 32];
    Acc acc[kDotGroup];
#pragma unroll
    for (int j = 0; j < kDotGroup; ++j) acc[j] = Acc(0);
    // one 4-value record per thread and step: all cnt + 1 vector loads are
    // issued before the first product (up to 9 loads in flight per thread;
    // with the products between the loads, the loads waited one by one)
    // (FP64 vectors, twice the registers per record and bound by the FP64
    // pipe, keep the loads next to their products)
    GRID_STRIDE(i, len4)
    {
        const vec4<T> wi = ld4(w + i);
        if constexpr (sizeof(T) == 4) {
            vec4<T> v[kDotGroup];
#pragma unroll
            for (int j = 0; j < kDotGroup; ++j)
                if (j < cnt)
                    v[j] = ld4((k0 + j == self_k ? w : V + (int64_t)(k0 + j) * vstride) + i);
                else
                    v[j] = vec4<T>{T(0), T(0), T(0), T(0)};
            // vectors j and j + 1 on the two halves of the paired
            // instructions (a missing j + 1 sums zeros, unused)
#pragma unroll
            for (int j = 0; j < kDotGroup; j += 2)
                if (j < cnt) {
                    Comp2 a2{make_float2(acc[j].s, acc[j + 1].s),
                             make_float2(acc[j].c, acc[j + 1].c)};
                    dot_acc2(a2, make_float2(v[j].x, v[j + 1].x), make_float2(wi.x, wi.x));
                    dot_acc2(a2, make_float2(v[j].y, v[j + 1].y), make_float2(wi.y, wi.y));
                    dot_acc2(a2, make_float2(v[j].z, v[j + 1].z), make_float2(wi.z, wi.z));
                    dot_acc2(a2, make_float2(v[j].w, v[j + 1].w), make_float2(wi.w, wi.w));
                    dot_renorm2(a2);
                    acc[j].s = a2.s.x;
                    acc[j].c = a2.c.x;
                    acc[j + 1].s = a2.s.y;
                    acc[j + 1].c = a2.c.y;
                }
        } else {
#pragma unroll
            for (int j = 0; j < kDotGroup; ++j)
                if (j < cnt) {
                    const vec4<T> v =
                        k0 + j == self_k ? wi : ld4(V + (int64_t)(k0 + j) * vstride + i);
                    dot_acc(acc[j], v.x, wi.x);
                    dot_acc(acc[j], v.y, wi.y);
                    dot_acc(acc[j], v.z, wi.z);
                    dot_acc(acc[j], v.w, wi.w);
                    dot_renorm(acc[j]);
                }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kDotGroup; ++j) {
        double v = dot_value(acc[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double v = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) v += red[threadIdx.x][q];
        partial[(int64_t)(k0 + threadIdx.x) * kRedGrid + blockIdx.x] = v;
    }
}

// out[k] (+)= sum_b partial[k][b] for k < cnt; one block per k, fixed tree.
// mode 0: store, 1: add, 2: store sqrt (norm)
// (nb partials per k, rows kRedGrid apart)
__global__ void multi_dot_final_kernel(int cnt, const double *partial, double *out, int mode,
                                       const double *cond = nullptr, int nb = kRedGrid)
{
    if (cond && *cond == 0.0) return;
    __shared__ double red[kRedThreads];
    const int k = blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partial[(int64_t)k * kRedGrid + b];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (mode == 0) out[k] = red[0];
        else if (mode == 1) out[k] += red[0];
        else out[k] = sqrt(red[0]);
    }
    (void)cnt;
}

// w_i -= sum_k V_k[i] h[k], k < cnt: FP64 vectors in FP64; FP32 vectors
// (the mixed mode's Krylov basis) with FP32 FMAs and h rounded to FP32.  One
// 4-value record per thread and step, four basis vectors loaded ahead of their
// FMAs (the FMA order per entry is k = 0, 1, 2, ...).  With norm_partial the
// same pass sums |w_new|^2 (like the dots: FP64, or exact FP32 products in
// double-float) per CTA into norm_partial[block] (launch on the fixed
// kAxpyGrid x kRedThreads grid); with cond, nothing happens when *cond is 0.
constexpr int kMaxAxpy = 256;
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    multi_axpy_kernel(int cnt, int64_t len4, const vec4<T> *V, int64_t vstride, const double *h,
                      vec4<T> *w, double *norm_partial, const double *cond)
{
    if (cond && *cond == 0.0) return;
    using Acc = typename DotAcc<T>::type;
    Acc nacc = Acc(0);
    __shared__ double red[kRedThreads / 32];
    __shared__ T hs[kMaxAxpy];
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) hs[k] = (T)h[k];
    __syncthreads();
    GRID_STRIDE(i, len4)
    {
        vec4<T> acc = w[i];
        int k = 0;
        for (; k + 4 <= cnt; k += 4) {
            vec4<T> v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = ld4(V + (int64_t)(k + q) * vstride + i);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T hk = hs[k + q];
                acc.x = fma_rn(-v[q].x, hk, acc.x);
                acc.y = fma_rn(-v[q].y, hk, acc.y);
                acc.z = fma_rn(-v[q].z, hk, acc.z);
                acc.w = fma_rn(-v[q].w, hk, acc.w);
            }
        }
        for (; k < cnt; ++k) {
            const vec4<T> v = ld4(V + (int64_t)k * vstride + i);
            const T hk = hs[k];
            acc.x = fma_rn(-v.x, hk, acc.x);
            acc.y = fma_rn(-v.y, hk, acc.y);
            acc.z = fma_rn(-v.z, hk, acc.z);
            acc.w = fma_rn(-v.w, hk, acc.w);
        }
        w[i] = acc;
        if (norm_partial) {
            dot_acc(nacc, acc.x, acc.x);
            dot_acc(nacc, acc.y, acc.y);
            dot_acc(nacc, acc.z, acc.z);
            dot_acc(nacc, acc.w, acc.w);
            dot_renorm(nacc);
        }
    }
    if (norm_partial) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        double v = dot_value(nacc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < kRedThreads / 32; ++q) t += red[q];
            norm_partial[blockIdx.x] = t;
        }
    }
}

// Kahan's test on the device: flag = 1 when |h[0..j]|^2 > |w|^2 / 2 (w . w in
// h[j + 1]), i.e. the classical Gram-Schmidt pass lost orthogonality and a
// second pass is due; lanes sum in a fixed order
__global__ void kahan_flag_kernel(int j, const double *h, double *flag)
{
    double v = 0.0;
    for (int i = threadIdx.x; i <= j; i += 32) v += h[i] * h[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *flag = (v <= 0.5 * h[j + 1]) ? 0.0 : 1.0;
}

__global__ void add_if_kernel(int n, const double *x, double *y, const double *cond)
{
    if (*cond == 0.0) return;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] += x[i];
}

// y = x / *den (0 when the norm vanished: lucky breakdown), in the vector's
// own precision (the scale is rounded once; GB300's FP64 unit is ~70x slower)
// (len a multiple of 4: one 4-value record per thread and step)
template <typename T>
__global__ void scale_by_inv_kernel(int64_t len, const double *den, const T *x, T *y)
{
    const double d = *den;
    const T s = (T)(d > 0.0 ? 1.0 / d : 0.0);
    const vec4<T> *x4 = (const vec4<T> *)x;
    vec4<T> *y4 = (vec4<T> *)y;
    GRID_STRIDE(i, len / 4)
    {
        vec4<T> v = ld4(x4 + i);
        v.x *= s;
        v.y *= s;
        v.z *= s;
        v.w *= s;
        y4[i] = v;
    }
}

// ------------------------------------------------------------ block Jacobi
__device__ __forceinline__ int node_color(int node, int NX1, int NY1)
{
    const int i = node % NX1, j = (node / NX1) % NY1, k = node / (NX1 * NY1);
    return (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
}

// colours: the node's entry of `colors` when given (tetrahedral meshes), else
// the parity colour of the structured grid
__device__ __forceinline__ int probe_color(int node, int NX1, int NY1, const int32_t *colors)
{
    return colors ? colors[node] : node_color(node, NX1, NY1);
}

template <typename T>
__global__ void probe_fill_kernel(int n, int NX1, int NY1, const int32_t *colors, int color,
                                  int comp, T *x)
{
    GRID_STRIDE(node, n)
    {
        const bool on = probe_color((int)node, NX1, NY1, colors) == color;
        for (int c = 0; c < 4; ++c) x[4 * node + c] = (on && c == comp) ? T(1) : T(0);
    }
}

template <typename T>
__global__ void probe_extract_kernel(int n, int NX1, int NY1, const int32_t *colors, int color,
                                     int comp, const T *Jx, T *blocks)
{
    GRID_STRIDE(node, n)
    if (probe_color((int)node, NX1, NY1, colors) == color)
        for (int r = 0; r < 4; ++r) blocks[16 * node + 4 * r + comp] = Jx[4 * node + r];
}

// Direct diagonal blocks, last step: the point masses' diagonal
// (cpl[node].x = D sum_B w_B N_a(xi_B)^2, or null) on the velocity diagonal,
// then the Dirichlet rows (mask) as unit rows, like the Jacobian's.
template <typename T>
__global__ void diag_finish_kernel(int64_t n, int ncols, const vec4<T> *cpl, const uint8_t *mask,
                                   T *blocks)
{
    GRID_STRIDE(node, n)
    {
        T *b = blocks + 16 * node;
        if (cpl) {
            const T d = cpl[node].x;
            for (int r = 0; r < 3; ++r) b[5 * r] += d;
        }
        if (mask)
            for (int r = 0; r < ncols; ++r)
                if (mask[4 * node + r])
                    for (int c = 0; c < ncols; ++c) b[4 * r + c] = r == c ? T(1) : T(0);
    }
}

// 4x4 inverse per node, Gauss-Jordan with partial pivoting in FP64; a
// singular block is replaced by the identity (no preconditioning there).
template <typename T> __global__ void block_invert_kernel(int n, const T *blocks, T *inv)
{
    GRID_STRIDE(node, n)
    {
        double a[4][8];
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                a[r][c] = (double)blocks[16 * node + 4 * r + c];
                a[r][4 + c] = r == c ? 1.0 : 0.0;
            }
        bool ok = true;
        for (int col = 0; col < 4 && ok; ++col) {
            int p = col;
            for (int r = col + 1; r < 4; ++r)
                if (fabs(a[r][col]) > fabs(a[p][col])) p = r;
            if (!(fabs(a[p][col]) > 0.0)) {
                ok = false;
                break;
            }
            if (p != col)
                for (int c = 0; c < 8; ++c) {
                    const double t = a[p][c];
                    a[p][c] = a[col][c];
                    a[col][c] = t;
                }
            const double piv = 1.0 / a[col][col];
            for (int c = 0; c < 8; ++c) a[col][c] *= piv;
            for (int r = 0; r < 4; ++r)
                if (r != col) {
                    const double f = a[r][col];
                    for (int c = 0; c < 8; ++c) a[r][c] -= f * a[col][c];
                }
        }
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c)
                inv[16 * node + 4 * r + c] = ok ? (T)a[r][4 + c] : (T)(r == c ? 1.0 : 0.0);
    }
}

template <typename T> __global__ void block_apply_kernel(int n, const T *inv, const T *x, T *y)
{
    GRID_STRIDE(node, n)
    {
        const T x0 = x[4 * node], x1 = x[4 * node + 1], x2 = x[4 * node + 2],
                x3 = x[4 * node + 3];
        const T *M = inv + 16 * node;
        for (int r = 0; r < 4; ++r)
            y[4 * node + r] = M[4 * r] * x0 + M[4 * r + 1] * x1 + M[4 * r + 2] * x2 +
                              M[4 * r + 3] * x3;
    }
}

// Schur-complement block preconditioner, velocity part: inverse of the 3x3
// velocity sub-block of each nodal block (Gauss-Jordan, partial pivoting,
// FP64), stored in the upper-left 3x3 of the node's 16 slots.
// Gauss-Jordan with partial pivoting in the blocks' own precision (an FP32
// preconditioner's inverse is stored in FP32 anyway; in FP64 the 2.1 M
// inversions at 128^3 took 366 us on GB300's FP64 unit)
template <typename T> __global__ void block_invert3_kernel(int n, const T *blocks, T *inv)
{
    GRID_STRIDE(node, n)
    {
        T a[3][6];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a[r][c] = blocks[16 * node + 4 * r + c];
                a[r][3 + c] = r == c ? T(1) : T(0);
            }
        bool ok = true;
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            if (!ok) break;
            int p = col;
#pragma unroll
            for (int r = col + 1; r < 3; ++r)
                if (fabs(a[r][col]) > fabs(a[p][col])) p = r;
            if (!(fabs(a[p][col]) > T(0))) {
                ok = false;
                break;
            }
            if (p != col)
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const T t = a[p][c];
                    a[p][c] = a[col][c];
                    a[col][c] = t;
                }
            const T piv = T(1) / a[col][col];
#pragma unroll
            for (int c = 0; c < 6; ++c) a[col][c] *= piv;
#pragma unroll
            for (int r = 0; r < 3; ++r)
                if (r != col) {
                    const T f = a[r][col];
#pragma unroll
                    for (int c = 0; c < 6; ++c) a[r][c] -= f * a[col][c];
                }
        }
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c)
                inv[16 * node + 4 * r + c] =
                    (r < 3 && c < 3) ? (ok ? a[r][3 + c] : (r == c ? T(1) : T(0))) : T(0);
    }
}

// Per box face f (x0, x1, y0, y1, z0, z1): cnt[f][0..3] = nodes inside the face
// (off its edges), of those with all three velocity components free, all
// nodes of the face, of those free.  Shared-memory sums per block, then one
// atomic per counter and block.
__global__ void face_count_kernel(int NX1, int NY1, int NZ1, const uint8_t *mask, int *cnt)
{
    __shared__ int c[24];
    if (threadIdx.x < 24) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = (int64_t)NX1 * NY1 * NZ1;
    const int dims[3] = {NX1 - 1, NY1 - 1, NZ1 - 1};
    GRID_STRIDE(node, n)
    {
        const int idx[3] = {(int)(node % NX1), (int)((node / NX1) % NY1),
                            (int)(node / ((int64_t)NX1 * NY1))};
        const bool fr = !mask || !(mask[4 * node] | mask[4 * node + 1] | mask[4 * node + 2]);
        for (int d = 0; d < 3; ++d)
            for (int side = 0; side < 2; ++side) {
                if (idx[d] != (side ? dims[d] : 0)) continue;
                bool inner = true;
                for (int e = 0; e < 3; ++e)
                    if (e != d) inner = inner && idx[e] > 0 && idx[e] < dims[e];
                int *cf = c + 4 * (2 * d + side);
                if (inner) {
                    atomicAdd(cf, 1);
                    if (fr) atomicAdd(cf + 1, 1);
                }
                atomicAdd(cf + 2, 1);
                if (fr) atomicAdd(cf + 3, 1);
            }
    }
    __syncthreads();
    if (threadIdx.x < 24 && c[threadIdx.x]) atomicAdd(cnt + threadIdx.x, c[threadIdx.x]);
}

// z_v = (3x3 velocity block)^{-1} v_v per node; the pressure entries are
// gathered into the contiguous right-hand side bp of the pressure V-cycle
template <typename T>
__global__ void schur_split_kernel(int n, const T *inv, const T *v, T *z, T *bp)
{
    GRID_STRIDE(node, n)
    {
        // vector loads of the node record and the block's three rows; z's
        // pressure slot is written by schur_merge_kernel afterwards
        const vec4<T> x = ld4((const vec4<T> *)v + node);
        const vec4<T> *M = (const vec4<T> *)(inv + 16 * node);
        vec4<T> zr;
        const vec4<T> m0 = ld4(M), m1 = ld4(M + 1), m2 = ld4(M + 2);
        zr.x = m0.x * x.x + m0.y * x.y + m0.z * x.z;
        zr.y = m1.x * x.x + m1.y * x.y + m1.z * x.z;
        zr.z = m2.x * x.x + m2.y * x.y + m2.z * x.z;
        zr.w = T(0);
        ((vec4<T> *)z)[node] = zr;
        bp[node] = x.w;
    }
}

// The GMRES basis scaling V = w / den fused with the Schur split of V for
// the next preconditioner application (the arithmetic of scale_by_inv_kernel
// and schur_split_kernel, one pass)
template <typename T>
__global__ void scale_split_kernel(int n, const double *den, const T *w, T *V, const T *inv, T *z,
                                   T *bp)
{
    const double dd = *den;
    const T sc = (T)(dd > 0.0 ? 1.0 / dd : 0.0);
    GRID_STRIDE(node, n)
    {
        vec4<T> x = ld4((const vec4<T> *)w + node);
        x.x *= sc;
        x.y *= sc;
        x.z *= sc;
        x.w *= sc;
        ((vec4<T> *)V)[node] = x;
        const vec4<T> *M = (const vec4<T> *)(inv + 16 * node);
        vec4<T> zr;
        const vec4<T> m0 = ld4(M), m1 = ld4(M + 1), m2 = ld4(M + 2);
        zr.x = m0.x * x.x + m0.y * x.y + m0.z * x.z;
        zr.y = m1.x * x.x + m1.y * x.y + m1.z * x.z;
        zr.z = m2.x * x.x + m2.y * x.y + m2.z * x.z;
        zr.w = T(0);
        ((vec4<T> *)z)[node] = zr;
        bp[node] = x.w;
    }
}

// z_p = V-cycle result / sigma, or z_p = v_p on Dirichlet pressure rows
template <typename T>
__global__ void schur_merge_kernel(int n, const T *v, const T *xp, const uint8_t *mask,
                                   T inv_sigma, T *z)
{
    GRID_STRIDE(node, n)
    z[4 * node + 3] = (mask && mask[4 * node + 3]) ? v[4 * node + 3] : xp[node] * inv_sigma;
}

// ------------------------------------------------------------ workspace
struct Work {
    int64_t n = 0, m = 0;
    int restart = 0;
    bool have = false;
    // FP64 state
    double *U = nullptr, *A = nullptr, *R = nullptr, *V1 = nullptr;
    double *pa = nullptr, *pv = nullptr, *prs = nullptr;  // [m][3]
    // working-precision buffers (8 bytes per entry so that either type fits)
    void *Uw = nullptr, *Aw = nullptr, *fw = nullptr, *xiw = nullptr, *ww = nullptr;
    void *pu = nullptr;                    // [m][3] point work
    double *bu = nullptr, *bv = nullptr, *ba = nullptr;  // solid stage values [m][3]
    void *buw = nullptr, *pw = nullptr;    // solid u_af and tangent output (working precision)
    void *Vk = nullptr;                    // [restart+1][4n]
    void *w = nullptr, *z = nullptr, *x = nullptr, *b = nullptr;
    void *blocks = nullptr, *inv = nullptr;  // [n][16]
    double *partial = nullptr;              // [restart+1][kRedGrid] + [kAxpyGrid]
    double *hcol = nullptr, *h2 = nullptr;  // [restart+2]
    double *hhost = nullptr;                // pinned
    int precond = 0;                        // 0 block-Jacobi, 1 Schur (pmg.cu)
    // the point-mass coupling of the Jacobian apply runs on a side stream
    // while the VMS Jacobian runs on the mesh's stream; its spread goes to
    // ftmp [n][4] (components 0..2), added to Jx after the join
    void *ftmp = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t reorth = 0;                     // second Gram-Schmidt passes taken
};

void free_work(Work &W)
{
    void *ptrs[] = {W.U, W.A, W.R, W.V1, W.pa, W.pv, W.prs, W.Uw, W.Aw, W.fw, W.xiw, W.ww, W.pu,
                    W.bu, W.bv, W.ba, W.buw, W.pw,
                    W.Vk, W.w, W.z, W.x, W.b, W.blocks, W.inv, W.partial, W.hcol, W.h2};
    for (void *p : ptrs) cudaFree(p);
    cudaFree(W.ftmp);
    if (W.side) cudaStreamDestroy(W.side);
    if (W.ev_fork) cudaEventDestroy(W.ev_fork);
    if (W.ev_join) cudaEventDestroy(W.ev_join);
    if (W.hhost) cudaFreeHost(W.hhost);
    W = Work();
}

}  // namespace

// The workspace lives in the mesh (one per mesh), behind an opaque pointer.
struct NewtonWorkspace {
    Work w;
};

void destroy_newton_workspace(fsi_mesh *m)
{
    if (m->newton) {
        free_work(m->newton->w);
        delete m->newton;
        m->newton = nullptr;
    }
}

namespace {

fsi_status ensure_work(fsi_mesh *mesh, int64_t m_pts, int restart)
{
    if (!mesh->newton) mesh->newton = new NewtonWorkspace();
    Work &W = mesh->newton->w;
    const int64_t n = mesh->n_nodes;
    if (W.have && W.n == n && W.m >= m_pts && W.restart >= restart) return FSI_OK;
    FSI_CUDA(cudaStreamSynchronize(mesh->stream), "sync");
    free_work(W);
    W.n = n;
    W.m = m_pts;
    W.restart = restart;
    const size_t v = (size_t)n * 4 * sizeof(double);
    const size_t pm = (size_t)(m_pts > 0 ? m_pts : 1) * 3 * sizeof(double);
    struct {
        void **p;
        size_t bytes;
    } req[] = {
        {(void **)&W.U, v}, {(void **)&W.A, v}, {(void **)&W.R, v}, {(void **)&W.V1, v},
        {(void **)&W.pa, pm}, {(void **)&W.pv, pm}, {(void **)&W.prs, pm},
        {&W.Uw, v}, {&W.Aw, v}, {&W.fw, v}, {&W.xiw, pm}, {&W.ww, pm / 3 + 8}, {&W.pu, pm},
        {(void **)&W.bu, pm}, {(void **)&W.bv, pm}, {(void **)&W.ba, pm}, {&W.buw, pm},
        {&W.pw, pm},
        {&W.Vk, v * (size_t)(restart + 1)}, {&W.w, v}, {&W.z, v}, {&W.x, v}, {&W.b, v},
        {&W.blocks, v * 4}, {&W.inv, v * 4}, {&W.ftmp, v},
        {(void **)&W.partial, ((size_t)(restart + 1) * kRedGrid + kAxpyGrid) * sizeof(double)},
        {(void **)&W.hcol, (size_t)(restart + 2) * sizeof(double)},
        {(void **)&W.h2, (size_t)(restart + 2) * sizeof(double)},
    };
    for (auto &r : req) {
        cudaError_t e = cudaMalloc(r.p, r.bytes);
        if (e != cudaSuccess) {
            free_work(W);
            return check_cuda(e, "Newton workspace allocation");
        }
    }
    cudaError_t e = cudaMallocHost((void **)&W.hhost, (size_t)(restart + 2) * sizeof(double));
    if (e != cudaSuccess) {
        free_work(W);
        return check_cuda(e, "pinned host buffer");
    }
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&W.side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W.ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W.ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_work(W);
        return check_cuda(e, "coupling side stream");
    }
    W.have = true;
    return FSI_OK;
}

template <typename T> fsi_prec prec_of() { return sizeof(T) == 8 ? FSI_F64 : FSI_F32; }

// ------------------------------------------------------------ operators
// FP64 coupled residual at st->y; leaves the FP64 stage in W.U, W.A.
// prec: FSI_F64 (native FP64) or FSI_DF64 (double-float VMS and coupling
// arithmetic on FP64 arrays, FP64-accurate to ~1e-14); stage and solid force in FP64
// R += the point masses' spread forces (no hyperelastic body), then the
// Dirichlet rows R = y - y_D; coupling in prec
fsi_status point_mass_residual_add(fsi_mesh *mesh, const fsi_step_state *st, double *R,
                                   fsi_prec prec)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t n = mesh->n_nodes;
    if (st->m > 0) {
        velocity_next_kernel<<<grid1d(n), 256, 0, s>>>(n, mesh->phys.dt, mesh->gamma, st->y,
                                                      st->Vn, st->An, W.V1);
        FSI_TRY(check_launch("velocity_next kernel"));
        FSI_TRY(fsi_dlm_interp(mesh, prec, st->m, st->elem, st->xi, st->y, W.pa));
        FSI_TRY(fsi_dlm_interp(mesh, prec, st->m, st->elem, st->xi, W.V1, W.pv));
        solid_force_kernel<<<grid1d(st->m), 256, 0, s>>>(
            st->m, st->elem, W.pa, W.pv, st->drho_s, st->k_s * mesh->phys.dt, st->g_s[0],
            st->g_s[1], st->g_s[2], W.prs);
        FSI_TRY(check_launch("solid force kernel"));
        FSI_TRY(fsi_dlm_spread(mesh, prec, st->m, st->elem, st->xi, st->cell_start, st->perm,
                               W.prs, st->w, R, 1));
    }
    if (st->mask) {
        dirichlet_residual_kernel<<<grid1d(4 * n), 256, 0, s>>>(4 * n, st->mask, st->y, st->yD, R);
        FSI_TRY(check_launch("dirichlet residual kernel"));
    }
    return FSI_OK;
}

fsi_status coupled_residual_impl(fsi_mesh *mesh, const fsi_step_state *st, double *R,
                                 fsi_prec prec = FSI_F64)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t n = mesh->n_nodes;
    FSI_TRY(fsi_stage(mesh, FSI_F64, st->y, st->Vn, st->An, st->s, W.U, W.A));
    FSI_TRY(vms_residual(mesh, prec, W.U, W.A, st->f, R));
    if (st->m > 0 && st->body) {
        // hyperelastic body: uddot_{n+1} = C^T Vdot_{n+1} at its nodes, stage
        // values, nodal residual R^s, spread without weights
        FSI_TRY(fsi_dlm_interp(mesh, prec, st->m, st->elem, st->xi, st->y, W.pa));
        FSI_TRY(solid_stage_impl(st->body, st->us, st->vs, st->as, W.pa, W.bu, W.bv, W.ba));
        FSI_TRY(solid_residual_impl(st->body, W.bu, W.bv, W.ba, st->us, st->g_s, W.prs));
        FSI_TRY(fsi_dlm_spread(mesh, prec, st->m, st->elem, st->xi, st->cell_start, st->perm,
                               W.prs, nullptr, R, 1));
        if (st->mask) {
            dirichlet_residual_kernel<<<grid1d(4 * n), 256, 0, s>>>(4 * n, st->mask, st->y, st->yD,
                                                                    R);
            FSI_TRY(check_launch("dirichlet residual kernel"));
        }
        return FSI_OK;
    }
    return point_mass_residual_add(mesh, st, R, prec);
}

// Working-precision copies of the linearisation point (after a residual).
template <typename T> fsi_status prepare_linearisation(fsi_mesh *mesh, const fsi_step_state *st)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t n4 = 4 * mesh->n_nodes;
    cast_kernel<double, T><<<grid1d(n4), 256, 0, s>>>(n4, W.U, (T *)W.Uw);
    cast_kernel<double, T><<<grid1d(n4), 256, 0, s>>>(n4, W.A, (T *)W.Aw);
    if (st->f) cast_kernel<double, T><<<grid1d(n4), 256, 0, s>>>(n4, st->f, (T *)W.fw);
    if (st->m > 0) {
        cast_kernel<double, T><<<grid1d(3 * st->m), 256, 0, s>>>(3 * st->m, st->xi, (T *)W.xiw);
        if (st->body)
            cast_kernel<double, T><<<grid1d(3 * st->m), 256, 0, s>>>(3 * st->m, W.bu, (T *)W.buw);
        if (st->w) cast_kernel<double, T><<<grid1d(st->m), 256, 0, s>>>(st->m, st->w, (T *)W.ww);
    }
    return check_launch("linearisation casts");
}

template <typename T>
fsi_status coupled_jacobian_impl(fsi_mesh *mesh, const fsi_step_state *st, const T *x, T *Jx)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t n = mesh->n_nodes;
    const fsi_prec P = prec_of<T>();
    // point masses on a structured grid: the coupling overlaps the VMS Jacobian
    const bool overlap = st->m > 0 && !st->body && !mesh->tet;
    if (overlap) {
        // x is ready on s: the side stream may start the coupling
        FSI_CUDA(cudaEventRecord(W.ev_fork, s), "event record");
        FSI_CUDA(cudaStreamWaitEvent(W.side, W.ev_fork, 0), "stream wait");
    }
    FSI_TRY(vms_jacobian(mesh, P, W.Uw, W.Aw, st->f ? W.fw : nullptr, x, Jx));
    if (st->m > 0 && st->body) {
        FSI_TRY(fsi_dlm_interp(mesh, P, st->m, st->elem, W.xiw, x, W.pu));
        FSI_TRY(solid_tangent_impl<T>(st->body, (const T *)W.buw, st->us, (const T *)W.pu,
                                      (T *)W.pw));
        FSI_TRY(fsi_dlm_spread(mesh, P, st->m, st->elem, W.xiw, st->cell_start, st->perm, W.pw,
                               nullptr, Jx, 1));
    } else if (st->m > 0 && !overlap) {
        FSI_TRY(fsi_dlm_interp(mesh, P, st->m, st->elem, W.xiw, x, W.pu));
        const double D = st->drho_s + st->k_s * mesh->gamma * mesh->phys.dt * mesh->phys.dt;
        scale_kernel<T><<<grid1d(3 * st->m), 256, 0, s>>>(3 * st->m, (T)D, (const T *)W.pu,
                                                        (T *)W.pu);
        FSI_TRY(check_launch("scale kernel"));
        FSI_TRY(fsi_dlm_spread(mesh, P, st->m, st->elem, W.xiw, st->cell_start, st->perm, W.pu,
                               st->w ? W.ww : nullptr, Jx, 1));
    } else if (st->m > 0) {
        // C D C^T x on the side stream (D = w (drho + k gamma dt^2)): it needs
        // only x, so it overlaps the VMS Jacobian issued above on s
        const double D = st->drho_s + st->k_s * mesh->gamma * mesh->phys.dt * mesh->phys.dt;
        mesh->stream = W.side;
        const fsi_status cs = [&]() -> fsi_status {
            FSI_TRY(fsi_dlm_interp(mesh, P, st->m, st->elem, W.xiw, x, W.pu));
            scale_kernel<T><<<grid1d(3 * st->m), 256, 0, W.side>>>(3 * st->m, (T)D,
                                                                  (const T *)W.pu, (T *)W.pu);
            FSI_TRY(check_launch("scale kernel"));
            return fsi_dlm_spread(mesh, P, st->m, st->elem, W.xiw, st->cell_start, st->perm,
                                  W.pu, st->w ? W.ww : nullptr, W.ftmp, 0);
        }();
        mesh->stream = s;
        FSI_TRY(cs);
        FSI_CUDA(cudaEventRecord(W.ev_join, W.side), "event record");
        FSI_CUDA(cudaStreamWaitEvent(s, W.ev_join, 0), "stream wait");
        if (st->mask && (reinterpret_cast<uintptr_t>(st->mask) & 3) == 0) {
            // the coupling's forces and the Dirichlet rows in one pass
            add_xyz_rows_kernel<T><<<grid1d(n), 256, 0, s>>>(
                n, (const vec4<T> *)W.ftmp, (const uchar4 *)st->mask, (const vec4<T> *)x,
                (vec4<T> *)Jx);
            return check_launch("coupling add kernel");
        }
        add_xyz_kernel<T><<<grid1d(n), 256, 0, s>>>(n, (const vec4<T> *)W.ftmp, (vec4<T> *)Jx);
        FSI_TRY(check_launch("coupling add kernel"));
    }
    if (st->mask) {
        dirichlet_rows_kernel<T><<<grid1d(4 * n), 256, 0, s>>>(4 * n, st->mask, x, Jx);
        FSI_TRY(check_launch("dirichlet rows kernel"));
    }
    return FSI_OK;
}

template <typename T>
fsi_status build_block_jacobi(fsi_mesh *mesh, const fsi_step_state *st, int precond)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int n = (int)mesh->n_nodes;
    const int NX1 = mesh->grid.N[0] + 1, NY1 = mesh->grid.N[1] + 1;
    T *px = (T *)W.z, *pj = (T *)W.w;
    // the Schur preconditioner needs only the 3x3 velocity blocks
    const int ncomp = precond == 1 ? 3 : 4;
    // 8 parity colours on the structured grid; a distance-2 colouring on a
    // tetrahedral mesh
    int ncolors = 8;
    const int32_t *colors = nullptr;
    if (mesh->tet) colors = tet_colors(mesh->tet, &ncolors);
    // uniform grid without a hyperelastic body: the blocks from their
    // definition (diag.cu), the point masses' diagonal by a squared spread;
    // otherwise by probing the coupled Jacobian
    const bool direct = !mesh->tet && !mesh->coords64 && !(st->m > 0 && st->body);
    if (direct) {
        FSI_TRY(vms_diag_blocks(mesh, prec_of<T>(), ncomp, W.Uw, W.Aw, st->f ? W.fw : nullptr,
                                W.blocks));
        const vec4<T> *cpl = nullptr;
        if (st->m > 0) {
            const double D = st->drho_s + st->k_s * mesh->gamma * mesh->phys.dt * mesh->phys.dt;
            FSI_TRY(spread_mass_diag<T>(mesh, st->m, (const T *)W.xiw, st->cell_start, st->perm,
                                        st->w ? (const T *)W.ww : nullptr, D, (T *)W.ftmp));
            cpl = (const vec4<T> *)W.ftmp;
        }
        diag_finish_kernel<T><<<grid1d(n), 256, 0, s>>>(n, ncomp, cpl, st->mask, (T *)W.blocks);
        FSI_TRY(check_launch("diagonal blocks finish"));
        ncolors = 0;  // no probing
    }
    for (int color = 0; color < ncolors; ++color)
        for (int comp = 0; comp < ncomp; ++comp) {
            probe_fill_kernel<T><<<grid1d(n), 256, 0, s>>>(n, NX1, NY1, colors, color, comp, px);
            FSI_TRY(check_launch("probe fill"));
            FSI_TRY(coupled_jacobian_impl<T>(mesh, st, px, pj));
            probe_extract_kernel<T><<<grid1d(n), 256, 0, s>>>(n, NX1, NY1, colors, color, comp,
                                                             pj, (T *)W.blocks);
            FSI_TRY(check_launch("probe extract"));
        }
    if (precond == 1) {
        block_invert3_kernel<T><<<grid1d(n), 256, 0, s>>>(n, (const T *)W.blocks, (T *)W.inv);
        FSI_TRY(check_launch("block invert"));
        // tetrahedral mesh: the algebraic multigrid eliminates boundary nodes
        // with free velocity and nodes with fixed pressure
        if (uses_amg(mesh)) return amg_set_from_mask(mesh, st->mask);
        // faces where the velocity is free (more than half of the face's inner
        // nodes, or of all its nodes when it has none inside) get Dirichlet
        // pressure in the Schur approximation
        int *cnt = (int *)W.partial;
        FSI_CUDA(cudaMemsetAsync(cnt, 0, 24 * sizeof(int), s), "memset");
        face_count_kernel<<<grid1d(n), 256, 0, s>>>(NX1, NY1, mesh->grid.N[2] + 1, st->mask, cnt);
        FSI_TRY(check_launch("face count"));
        int h[24];
        FSI_CUDA(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s), "memcpy");
        FSI_CUDA(cudaStreamSynchronize(s), "sync");
        int faces[6];
        for (int f = 0; f < 6; ++f) {
            const int *c = h + 4 * f;
            faces[f] = c[0] > 0 ? (2 * c[1] > c[0]) : (2 * c[3] > c[2]);
        }
        return pmg_set_faces(mesh, faces);
    }
    block_invert_kernel<T><<<grid1d(n), 256, 0, s>>>(n, (const T *)W.blocks, (T *)W.inv);
    return check_launch("block invert");
}

// ------------------------------------------------------------ Krylov helpers
// out[k] = V_k . w for k < cnt (with self_k: out[self_k] = w . w)
template <typename T>
fsi_status multi_dot(fsi_mesh *mesh, int cnt, const T *V, int64_t ld, const T *w, double *out,
                     int mode, int self_k = -1, const double *cond = nullptr)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t len = 4 * mesh->n_nodes;
    for (int k0 = 0; k0 < cnt; k0 += kDotGroup) {
        const int c = cnt - k0 < kDotGroup ? cnt - k0 : kDotGroup;
        multi_dot_partial_kernel<T><<<kRedGrid, kRedThreads, 0, s>>>(
            k0, c, len / 4, (const vec4<T> *)V, ld / 4, (const vec4<T> *)w, W.partial, self_k,
            cond);
    }
    FSI_TRY(check_launch("multi-dot partial"));
    multi_dot_final_kernel<<<cnt, kRedThreads, 0, s>>>(cnt, W.partial, out, mode, cond);
    return check_launch("multi-dot final");
}

// w -= V[:, :cnt] h (vectors of len = 4n entries, 16/32-byte aligned records);
// with norm_partial also the CTA partial sums of |w|^2 (fixed grid); with
// cond only when the device flag is set
template <typename T>
void multi_axpy(cudaStream_t s, int cnt, int64_t len, const T *V, int64_t ld, const double *h,
                T *w, double *norm_partial = nullptr, const double *cond = nullptr)
{
    multi_axpy_kernel<T><<<kAxpyGrid, kRedThreads, 0, s>>>(cnt, len / 4, (const vec4<T> *)V,
                                                          ld / 4, h, (vec4<T> *)w, norm_partial,
                                                          cond);
}

template <typename T> fsi_status norm2(fsi_mesh *mesh, const T *x, double *dev_out)
{
    return multi_dot<T>(mesh, 1, x, 0, x, dev_out, 2);
}

fsi_status host_scalar(fsi_mesh *mesh, const double *dev, double *out)
{
    Work &W = mesh->newton->w;
    FSI_CUDA(cudaMemcpyAsync(W.hhost, dev, sizeof(double), cudaMemcpyDeviceToHost, mesh->stream),
             "memcpy");
    FSI_CUDA(cudaStreamSynchronize(mesh->stream), "sync");
    *out = W.hhost[0];
    return FSI_OK;
}

// out = M^{-1} in: nodal 4x4 block-Jacobi (precond 0), or the block-diagonal
// Schur-complement preconditioner (precond 1): 3x3 velocity blocks and
// sigma^{-1} x one pressure V-cycle, sigma = alpha_f gamma dt / (alpha_m rho);
// in and out must not alias (the split writes all of out's records before the
// merge reads in's pressure slots)
template <typename T>
// (presplit: scale_split_kernel has already written out's velocity slots and
// the V-cycle's right-hand side from `in`)
fsi_status apply_precond(fsi_mesh *mesh, const fsi_step_state *st, const T *in, T *out,
                         bool presplit = false)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int n = (int)mesh->n_nodes;
    if (W.precond == 0) {
        block_apply_kernel<T><<<grid1d(n), 256, 0, s>>>(n, (const T *)W.inv, in, out);
        return check_launch("block apply");
    }
    const bool amg = uses_amg(mesh);
    T *bp = (T *)(amg ? amg_fine_buffer(mesh, 0) : pmg_fine_buffer(mesh, 0));
    T *xp = (T *)(amg ? amg_fine_buffer(mesh, 1) : pmg_fine_buffer(mesh, 1));
    if (!presplit) {
        schur_split_kernel<T><<<grid1d(n), 256, 0, s>>>(n, (const T *)W.inv, in, out, bp);
        FSI_TRY(check_launch("Schur split"));
    }
    const double sigma = mesh->alpha_f * mesh->gamma * mesh->phys.dt / (mesh->alpha_m * mesh->phys.rho);
    if (!amg) {
        // the V-cycle's last smoothing step writes z_p itself (no merge pass)
        bool done = false;
        FSI_TRY(pmg_vcycle_schur<T>(mesh, bp, out, in, st->mask, (T)(1.0 / sigma), &done));
        if (done) return FSI_OK;
    }
    FSI_TRY(amg ? amg_vcycle<T>(mesh, bp, xp) : pmg_vcycle<T>(mesh, bp, xp));
    schur_merge_kernel<T><<<grid1d(n), 256, 0, s>>>(n, in, xp, st->mask, (T)(1.0 / sigma), out);
    return check_launch("Schur merge");
}

// GMRES(restart) with right preconditioning M^{-1} (block Jacobi) on
// J x = b, x0 = 0, to ||b - J x|| <= rtol ||b||.  Result in W.x.
template <typename T>
fsi_status gmres(fsi_mesh *mesh, const fsi_step_state *st, int restart, int max_its, double rtol,
                 int *its_out)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t len = 4 * mesh->n_nodes;
    T *V = (T *)W.Vk, *w = (T *)W.w, *z = (T *)W.z, *x = (T *)W.x, *b = (T *)W.b;
    const int64_t ld = len;
    std::vector<double> H((size_t)(restart + 1) * restart, 0.0), cs(restart), sn(restart),
        g(restart + 1), y(restart);
    zero_kernel<T><<<grid1d(len), 256, 0, s>>>(len, x);
    FSI_TRY(check_launch("zero"));
    // r = b (x0 = 0)
    cudaMemcpyAsync(w, b, len * sizeof(T), cudaMemcpyDeviceToDevice, s);
    double beta = 0.0, beta0 = 0.0;
    FSI_TRY(norm2<T>(mesh, w, W.hcol));
    FSI_TRY(host_scalar(mesh, W.hcol, &beta));
    beta0 = beta;
    int its = 0;
    if (!(beta > 0.0)) {
        *its_out = 0;
        return std::isfinite(beta) ? FSI_OK : set_error(FSI_ERR_NAN, "GMRES: non-finite rhs");
    }
    const double target = rtol * beta0;
    // with the geometric-multigrid Schur preconditioner every basis vector's
    // scaling also does its Schur split for the next iteration
    const bool fuse = W.precond != 0 && !uses_amg(mesh);
    T *bp = nullptr;
    if (fuse) {
        FSI_TRY(pmg_ensure(mesh));
        bp = (T *)pmg_fine_buffer(mesh, 0);
    }
    auto scale_basis = [&](const double *den, T *dst) {
        if (fuse)
            scale_split_kernel<T><<<grid1d(len / 4), 256, 0, s>>>(
                (int)(len / 4), den, w, dst, (const T *)W.inv, z, bp);
        else
            scale_by_inv_kernel<T><<<grid1d(len), 256, 0, s>>>(len, den, w, dst);
    };
    while (true) {
        scale_basis(W.hcol, V);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jj = 0;
        bool done = false;
        for (int j = 0; j < restart && its < max_its; ++j) {
            T *Vj = V + (int64_t)j * ld;
            FSI_TRY(apply_precond<T>(mesh, st, Vj, z, fuse));
            FSI_TRY(coupled_jacobian_impl<T>(mesh, st, z, w));
            // classical Gram-Schmidt, h = V^T w (and |w|^2 in the same pass), with
            // a second pass only when Kahan's criterion flags a loss of
            // orthogonality: |h|^2 > |w|^2 / 2, i.e. |w - V h| < |w| / sqrt(2)
            // Kahan's test runs on the device and the second pass (when it is
            // due) is launched conditionally, so the iteration needs one host
            // synchronisation, at its end; |w|^2 of the orthogonalised vector is
            // summed by the update pass itself
            double *flag = W.h2 + restart + 1;
            double *npart = W.partial + (int64_t)(restart + 1) * kRedGrid;
            FSI_TRY(multi_dot<T>(mesh, j + 2, V, ld, w, W.hcol, 0, j + 1));
            kahan_flag_kernel<<<1, 32, 0, s>>>(j, W.hcol, flag);
            multi_axpy<T>(s, j + 1, len, V, ld, W.hcol, w, npart);
            FSI_TRY(multi_dot<T>(mesh, j + 1, V, ld, w, W.h2, 0, -1, flag));
            multi_axpy<T>(s, j + 1, len, V, ld, W.h2, w, npart, flag);
            add_if_kernel<<<1, 64, 0, s>>>(j + 1, W.h2, W.hcol, flag);
            multi_dot_final_kernel<<<1, kRedThreads, 0, s>>>(1, npart, W.hcol + j + 1, 2, nullptr,
                                                             kAxpyGrid);
            FSI_TRY(check_launch("Gram-Schmidt"));
            scale_basis(W.hcol + j + 1, V + (int64_t)(j + 1) * ld);
            FSI_CUDA(cudaMemcpyAsync(W.hhost, W.hcol, (j + 2) * sizeof(double),
                                     cudaMemcpyDeviceToHost, s),
                     "memcpy");
            FSI_CUDA(cudaMemcpyAsync(W.hhost + j + 2, flag, sizeof(double),
                                     cudaMemcpyDeviceToHost, s),
                     "memcpy");
            FSI_CUDA(cudaStreamSynchronize(s), "GMRES sync");
            if (W.hhost[j + 2] != 0.0) ++W.reorth;
            ++its;
            double *h = &H[(size_t)j * (restart + 1)];
            for (int i = 0; i <= j + 1; ++i) h[i] = W.hhost[i];
            if (!std::isfinite(h[j + 1]))
                return set_error(FSI_ERR_NAN, "GMRES: non-finite Arnoldi coefficient");
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * h[i] + sn[i] * h[i + 1];
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = t;
            }
            const double r = std::hypot(h[j], h[j + 1]);
            cs[j] = r > 0.0 ? h[j] / r : 1.0;
            sn[j] = r > 0.0 ? h[j + 1] / r : 0.0;
            h[j] = r;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jj = j + 1;
            if (std::fabs(g[j + 1]) <= target || W.hhost[j + 1] == 0.0) {
                done = true;
                break;
            }
        }
        // back substitution and x += M^{-1} V y
        for (int i = jj - 1; i >= 0; --i) {
            double t = g[i];
            for (int k = i + 1; k < jj; ++k) t -= H[(size_t)k * (restart + 1) + i] * y[k];
            const double d = H[(size_t)i * (restart + 1) + i];
            y[i] = d != 0.0 ? t / d : 0.0;
        }
        for (int i = 0; i < jj; ++i) W.hhost[i] = -y[i];
        FSI_CUDA(cudaMemcpyAsync(W.h2, W.hhost, jj * sizeof(double), cudaMemcpyHostToDevice, s),
                 "memcpy");
        zero_kernel<T><<<grid1d(len), 256, 0, s>>>(len, w);
        multi_axpy<T>(s, jj, len, V, ld, W.h2, w);  // w = -V (-y)
        FSI_TRY(apply_precond<T>(mesh, st, w, z));
        add_kernel<T><<<grid1d(len), 256, 0, s>>>(len, z, x);
        FSI_TRY(check_launch("GMRES update"));
        if (done || its >= max_its) break;
        // restart: r = b - J x
        FSI_TRY(coupled_jacobian_impl<T>(mesh, st, x, z));
        sub_kernel<T><<<grid1d(len), 256, 0, s>>>(len, b, z, w);
        FSI_TRY(norm2<T>(mesh, w, W.hcol));
        FSI_TRY(host_scalar(mesh, W.hcol, &beta));
        if (!std::isfinite(beta)) return set_error(FSI_ERR_NAN, "GMRES: non-finite residual");
        if (beta <= target) break;
    }
    *its_out = its;
    return FSI_OK;
}

template <typename T>
fsi_status newton_impl(fsi_mesh *mesh, const fsi_newton_opts *o, const fsi_step_state *st,
                       fsi_newton_report *rep)
{
    Work &W = mesh->newton->w;
    cudaStream_t s = mesh->stream;
    const int64_t len = 4 * mesh->n_nodes;
    const fsi_prec rp = o->residual_prec == FSI_DF64 ? FSI_DF64 : FSI_F64;
    if (o->R0 && !(st->m > 0 && st->body)) {
        // the caller's R(y_0); the linearisation still needs the stage values
        FSI_TRY(fsi_stage(mesh, FSI_F64, st->y, st->Vn, st->An, st->s, W.U, W.A));
        FSI_CUDA(cudaMemcpyAsync(W.R, o->R0, len * sizeof(double), cudaMemcpyDeviceToDevice, s),
                 "memcpy");
    } else {
        FSI_TRY(coupled_residual_impl(mesh, st, W.R, rp));
    }
    double r = 0.0;
    FSI_TRY(norm2<double>(mesh, W.R, W.hcol));
    FSI_TRY(host_scalar(mesh, W.hcol, &r));
    rep->r0 = r;
    rep->r_ref = o->r_ref > 0.0 ? o->r_ref : r;
    rep->r_final = r;
    if (!std::isfinite(r)) return set_error(FSI_ERR_NAN, "Newton: non-finite initial residual");
    const double target = o->newton_rtol * rep->r_ref;
    int it = 0;
    while (r > target && it < o->max_newton) {
        FSI_TRY(prepare_linearisation<T>(mesh, st));
        if (rep->precond_builds == 0 || (o->precond_every > 0 && it % o->precond_every == 0)) {
            FSI_TRY(build_block_jacobi<T>(mesh, st, o->precond));
            rep->precond_builds++;
        }
        neg_cast_kernel<T><<<grid1d(len), 256, 0, s>>>(len, W.R, (T *)W.b);
        // inexact Newton without oversolving: plan the fewest iterations n
        // whose linear reductions, each no tighter than the floor
        // krylov_rtol, reach half the absolute target from r, and ask this
        // solve for the n-th root of that reduction (n = 1: 0.5 target / r)
        const double need = 0.5 * target / r;
        double eta = o->krylov_rtol;
        if (need >= eta) {
            eta = need < 0.5 ? need : 0.5;
        } else if (o->krylov_rtol < 0.5) {
            const int nn = (int)std::ceil(std::log(need) / std::log(o->krylov_rtol) - 1e-9);
            const double root = std::pow(need, 1.0 / std::max(nn, 1));
            if (root > eta) eta = root;
        }
        int its = 0;
        FSI_TRY(gmres<T>(mesh, st, o->restart, o->max_krylov, eta, &its));
        rep->krylov_iters += its;
        add_to_f64_kernel<T><<<grid1d(len), 256, 0, s>>>(len, (const T *)W.x, st->y);
        FSI_TRY(check_launch("Newton update"));
        ++it;
        FSI_TRY(coupled_residual_impl(mesh, st, W.R, rp));
        FSI_TRY(norm2<double>(mesh, W.R, W.hcol));
        FSI_TRY(host_scalar(mesh, W.hcol, &r));
        rep->r_final = r;
        rep->newton_iters = it;
        if (!std::isfinite(r)) return set_error(FSI_ERR_NAN, "Newton: non-finite residual");
    }
    rep->converged = r <= target;
    if (!rep->converged)
        return set_error(FSI_ERR_NOCONV, "Newton: ||R|| = %.3e > %.3e after %d iterations", r,
                         target, it);
    return FSI_OK;
}

}  // namespace

// one linearisation at st->y (stage values, and for a hyperelastic body its
// stage values through the coupled residual), then J x_i for k FP32 vectors;
// with R_fit the residual at st->y too: the VMS part in FP32 from the
// linearisation's FP32 copies, the coupling and the Dirichlet rows
// double-float (a body's residual entirely double-float)
fsi_status coupled_jacobian_f32(fsi_mesh *mesh, const fsi_step_state *st, int k,
                                const float *const *x, float *const *Jx, double *R_fit)
{
    FSI_TRY(ensure_work(mesh, st->m, 1));
    Work &W = mesh->newton->w;
    const bool body = st->m > 0 && st->body;
    if (body) FSI_TRY(coupled_residual_impl(mesh, st, R_fit ? R_fit : W.R, R_fit ? FSI_DF64 : FSI_F64));
    else FSI_TRY(fsi_stage(mesh, FSI_F64, st->y, st->Vn, st->An, st->s, W.U, W.A));
    FSI_TRY(prepare_linearisation<float>(mesh, st));
    if (R_fit && !body) {
        const int64_t n4 = 4 * mesh->n_nodes;
        float *r32 = (float *)W.z;
        FSI_TRY(vms_residual(mesh, FSI_F32, W.Uw, W.Aw, st->f ? W.fw : nullptr, r32));
        cast_kernel<float, double><<<grid1d(n4), 256, 0, mesh->stream>>>(n4, r32, R_fit);
        FSI_TRY(check_launch("residual cast"));
        FSI_TRY(point_mass_residual_add(mesh, st, R_fit, FSI_DF64));
    }
    for (int i = 0; i < k; ++i) FSI_TRY(coupled_jacobian_impl<float>(mesh, st, x[i], Jx[i]));
    return FSI_OK;
}

namespace {

fsi_status validate_state(const fsi_mesh *mesh, const fsi_step_state *st)
{
    if (!st) return set_error(FSI_ERR_ARG, "state is NULL");
    if (!st->y || !st->Vn || !st->An) return set_error(FSI_ERR_ARG, "state: NULL y, Vn or An");
    if ((st->mask == nullptr) != (st->yD == nullptr))
        return set_error(FSI_ERR_ARG, "state: pass both mask and yD, or neither");
    if (st->m < 0 || st->m >= INT32_MAX) return set_error(FSI_ERR_ARG, "state: m out of range");
    if (st->m > 0 && (!st->elem || !st->xi || !st->cell_start || !st->perm))
        return set_error(FSI_ERR_ARG, "state: points need elem, xi, cell_start and perm");
    if (st->body) {
        if (st->m != solid_nodes(st->body))
            return set_error(FSI_ERR_ARG, "state: m must be the solid's node count");
        if (!st->us || !st->vs || !st->as)
            return set_error(FSI_ERR_ARG, "state: the solid needs us, vs and as");
    }
    (void)mesh;
    return FSI_OK;
}

}  // namespace

fsi_status validate_step_state(const fsi_mesh *mesh, const fsi_step_state *st)
{
    return validate_state(mesh, st);
}

}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status fsi_coupled_residual(fsi_mesh *mesh, fsi_prec prec, const fsi_step_state *st,
                                double *R)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(validate_state(mesh, st));
    if (!R) return set_error(FSI_ERR_ARG, "R is NULL");
    if (prec != FSI_F64 && prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "fsi_coupled_residual: precision must be FSI_F64 or FSI_DF64");
    FSI_DEVICE(mesh->device);
    FSI_TRY(ensure_work(mesh, st->m, 1));
    return coupled_residual_impl(mesh, st, R, prec);
}

fsi_status fsi_coupled_jacobian_apply(fsi_mesh *mesh, fsi_prec prec, const fsi_step_state *st,
                                      const void *x, void *Jx)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(validate_state(mesh, st));
    if (!x || !Jx || x == Jx) return set_error(FSI_ERR_ARG, "bad x / Jx");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(mesh->device);
    FSI_TRY(ensure_work(mesh, st->m, 1));
    Work &W = mesh->newton->w;
    FSI_TRY(coupled_residual_impl(mesh, st, W.R));
    if (prec == FSI_F64) {
        FSI_TRY(prepare_linearisation<double>(mesh, st));
        return coupled_jacobian_impl<double>(mesh, st, (const double *)x, (double *)Jx);
    }
    FSI_TRY(prepare_linearisation<float>(mesh, st));
    return coupled_jacobian_impl<float>(mesh, st, (const float *)x, (float *)Jx);
}

fsi_status fsi_block_diagonal(fsi_mesh *mesh, fsi_prec prec, const fsi_step_state *st,
                              void *blocks)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(validate_state(mesh, st));
    if (!blocks) return set_error(FSI_ERR_ARG, "blocks is NULL");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(mesh->device);
    FSI_TRY(ensure_work(mesh, st->m, 1));
    Work &W = mesh->newton->w;
    FSI_TRY(coupled_residual_impl(mesh, st, W.R));
    const size_t bytes = (size_t)mesh->n_nodes * 16 * (prec == FSI_F64 ? 8 : 4);
    if (prec == FSI_F64) {
        FSI_TRY(prepare_linearisation<double>(mesh, st));
        FSI_TRY(build_block_jacobi<double>(mesh, st, 0));
    } else {
        FSI_TRY(prepare_linearisation<float>(mesh, st));
        FSI_TRY(build_block_jacobi<float>(mesh, st, 0));
    }
    FSI_CUDA(cudaMemcpyAsync(blocks, W.blocks, bytes, cudaMemcpyDeviceToDevice, mesh->stream),
             "memcpy");
    return FSI_OK;
}

fsi_status fsi_newton_step(fsi_mesh *mesh, const fsi_newton_opts *opts, const fsi_step_state *st,
                           fsi_newton_report *report)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(validate_state(mesh, st));
    if (!opts || !report) return set_error(FSI_ERR_ARG, "opts or report is NULL");
    if (opts->restart < 1 || opts->restart > 200 || opts->max_newton < 0 ||
        opts->max_krylov < 1 || !(opts->newton_rtol > 0.0) || !(opts->krylov_rtol > 0.0) ||
        opts->precond < 0 || opts->precond > 1 ||
        (opts->residual_prec != FSI_F64 && opts->residual_prec != FSI_DF64))
        return set_error(FSI_ERR_ARG, "invalid Newton options");
    std::memset(report, 0, sizeof *report);
    const auto t0 = std::chrono::steady_clock::now();
    FSI_DEVICE(mesh->device);
    FSI_TRY(ensure_work(mesh, st->m, opts->restart));
    mesh->newton->w.precond = opts->precond;
    fsi_status stt = opts->mixed ? newton_impl<float>(mesh, opts, st, report)
                                 : newton_impl<double>(mesh, opts, st, report);
    cudaStreamSynchronize(mesh->stream);
    report->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return stt;
}

fsi_status fsi_multi_dot(int device, fsi_prec prec, int64_t len, int nvec, const void *V,
                         int64_t ldv, const void *w, double *out)
{
    if (!V || !w || !out) return set_error(FSI_ERR_ARG, "fsi_multi_dot: NULL argument");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    if (len < 4 || len % 4 != 0 || ldv < len || ldv % 4 != 0 || nvec < 1 || nvec > kMaxAxpy)
        return set_error(FSI_ERR_ARG, "fsi_multi_dot: bad sizes");
    const size_t esz = prec == FSI_F64 ? sizeof(double) : sizeof(float);
    if (((uintptr_t)V | (uintptr_t)w) % (4 * esz) != 0)
        return set_error(FSI_ERR_ARG, "fsi_multi_dot: V and w must be aligned to 4 entries");
    FSI_DEVICE(device);
    double *partial = nullptr;
    FSI_CUDA(cudaMallocAsync((void **)&partial, (size_t)nvec * kRedGrid * sizeof(double), 0),
             "partial sums");
    for (int k0 = 0; k0 < nvec; k0 += kDotGroup) {
        const int c = nvec - k0 < kDotGroup ? nvec - k0 : kDotGroup;
        if (prec == FSI_F64)
            multi_dot_partial_kernel<double><<<kRedGrid, kRedThreads, 0, 0>>>(
                k0, c, len / 4, (const vec4<double> *)V, ldv / 4, (const vec4<double> *)w, partial,
                -1, nullptr);
        else
            multi_dot_partial_kernel<float><<<kRedGrid, kRedThreads, 0, 0>>>(
                k0, c, len / 4, (const vec4<float> *)V, ldv / 4, (const vec4<float> *)w, partial,
                -1, nullptr);
    }
    multi_dot_final_kernel<<<nvec, kRedThreads, 0, 0>>>(nvec, partial, out, 0);
    const fsi_status st = check_launch("multi-dot kernels");
    cudaFreeAsync(partial, 0);
    return st;
}

fsi_status fsi_measure_blas1(int device, fsi_prec prec, int64_t len, int nvec, int reps,
                             double *dot_seconds, double *axpy_seconds)
{
    if (!dot_seconds || !axpy_seconds) return set_error(FSI_ERR_ARG, "NULL output");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    if (len < 4 || len % 4 != 0 || nvec < 1 || nvec > kMaxAxpy || reps < 1)
        return set_error(FSI_ERR_ARG, "fsi_measure_blas1: bad sizes");
    FSI_DEVICE(device);
    const size_t esz = prec == FSI_F64 ? sizeof(double) : sizeof(float);
    void *V = nullptr, *w = nullptr;
    double *partial = nullptr, *h = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fsi_status st = check_cuda(cudaMalloc(&V, (size_t)nvec * len * esz), "buffers");
    if (st == FSI_OK) st = check_cuda(cudaMalloc(&w, (size_t)len * esz), "buffers");
    if (st == FSI_OK)
        st = check_cuda(cudaMalloc(&partial, (size_t)(nvec + 1) * kRedGrid * sizeof(double)),
                        "buffers");
    if (st == FSI_OK) st = check_cuda(cudaMalloc(&h, (size_t)(nvec + 1) * sizeof(double)), "buffers");
    if (st == FSI_OK) st = check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    if (st == FSI_OK) st = check_cuda(cudaEventCreate(&e0), "event");
    if (st == FSI_OK) st = check_cuda(cudaEventCreate(&e1), "event");
    if (st == FSI_OK) st = check_cuda(cudaMemsetAsync(V, 0, (size_t)nvec * len * esz, s), "memset");
    if (st == FSI_OK) st = check_cuda(cudaMemsetAsync(w, 0, (size_t)len * esz, s), "memset");
    if (st == FSI_OK) st = check_cuda(cudaMemsetAsync(h, 0, (size_t)(nvec + 1) * sizeof(double), s),
                                      "memset");
    auto dots = [&]() {
        for (int k0 = 0; k0 < nvec; k0 += kDotGroup) {
            const int c = nvec - k0 < kDotGroup ? nvec - k0 : kDotGroup;
            if (prec == FSI_F64)
                multi_dot_partial_kernel<double><<<kRedGrid, kRedThreads, 0, s>>>(
                    k0, c, len / 4, (const vec4<double> *)V, len / 4, (const vec4<double> *)w,
                    partial, -1, nullptr);
            else
                multi_dot_partial_kernel<float><<<kRedGrid, kRedThreads, 0, s>>>(
                    k0, c, len / 4, (const vec4<float> *)V, len / 4, (const vec4<float> *)w,
                    partial, -1, nullptr);
        }
        multi_dot_final_kernel<<<nvec, kRedThreads, 0, s>>>(nvec, partial, h, 0);
    };
    auto axpy = [&]() {
        if (prec == FSI_F64)
            multi_axpy<double>(s, nvec, len, (const double *)V, len, h, (double *)w, partial);
        else
            multi_axpy<float>(s, nvec, len, (const float *)V, len, h, (float *)w, partial);
    };
    float ms = 0.f;
    for (int which = 0; st == FSI_OK && which < 2; ++which) {
        auto run = [&]() {
            if (which == 0) dots();
            else axpy();
        };
        run();
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) run();
        cudaEventRecord(e1, s);
        st = check_cuda(cudaEventSynchronize(e1), "BLAS-1 kernels");
        if (st == FSI_OK) st = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
        if (st == FSI_OK) (which == 0 ? *dot_seconds : *axpy_seconds) = 1e-3 * ms / reps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(V);
    cudaFree(w);
    cudaFree(partial);
    cudaFree(h);
    return st;
}

}  // extern "C"
