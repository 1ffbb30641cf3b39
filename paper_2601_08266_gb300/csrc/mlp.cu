// mlp.cu -- the learned initial guess (an extension; the paper has no
// counterpart): a 112 -> 256 -> 256 -> 4 ReLU network whose GEMMs run on the
// tensor cores in BF16 with FP32 accumulation, trained on the GPU by these
// kernels (forward, backward, Adam) and applied per node to predict the
// Newton predictor y^(0) = y_n + e + c, e = 2 d_{n-1} - d_{n-2}.
//
// GEMMs: the tcgen05 tensor-core kernel of mlp_gemm.cu (BF16 operands, FP32
// accumulation in TMEM, fused epilogues: bias, ReLU keeping the
// pre-activation, the ReLU mask of the backward pass).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fsi_internal.cuh"

struct fsi_mlp {
    int device;
    cudaStream_t stream;
    int64_t max_batch;
    // activations [max_batch] x {256, 256, 256, 256, 4, 4} and gradients
    float *Z1, *H1, *Z2, *H2, *O, *dO, *dZ1, *dZ2;
    float *X;       // features of a predict chunk [max_batch][112]
    double *loss_partial;
    void *packed;   // BF16 weights in the tensor-core operand layout (mlp_tc.cu)
    int *tc_err;    // wait-timeout flag of the tensor-core kernels (predict and GEMMs)
    float *gemm_work;  // split-K partial tiles of the weight-gradient GEMMs
};

namespace fsi {
namespace {

constexpr int NI = 112, NH = 256, NO = 4;
constexpr int64_t OFF_W1 = 0, OFF_b1 = OFF_W1 + NI * NH, OFF_W2 = OFF_b1 + NH,
                  OFF_b2 = OFF_W2 + NH * NH, OFF_W3 = OFF_b2 + NH, OFF_b3 = OFF_W3 + NH * NO,
                  N_PARAMS = OFF_b3 + NO;

enum Epi { EPI_STORE = TC_EPI_STORE, EPI_BIAS = TC_EPI_BIAS, EPI_BIAS_RELU = TC_EPI_BIAS_RELU,
           EPI_MASK = TC_EPI_MASK };

fsi_status gemm(const fsi_mlp *h, const TcGemm &g)
{
    return tc_gemm(h->stream, g, h->gemm_work, h->tc_err);
}

TcGemm ga(int M, int N, int K, const float *A, int64_t lda, int tA, const float *B, int64_t ldb,
          int tB, float *C, int64_t ldc, int epi = EPI_STORE, const float *bias = nullptr,
          float *Cpre = nullptr, const float *mask = nullptr)
{
    TcGemm g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.transA = tA;
    g.B = B; g.ldb = ldb; g.transB = tB;
    g.C = C; g.ldc = ldc; g.epi = epi; g.bias = bias; g.Cpre = Cpre; g.mask = mask;
    g.BN = 0;
    return g;
}

// dO = (O - T)/B; per-block partial sums of 1/2 |O - T|^2 / B (FP64)
__global__ void loss_kernel(int64_t B, const float *O, const float *T, float *dO,
                            double *partial)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B * NO;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = O[i] - T[i];
        dO[i] = d / (float)B;
        acc += 0.5 * (double)d * (double)d / (double)B;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void loss_final_kernel(int nb, const double *partial, float *loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partial[b];
        *loss = (float)s;
    }
}

// db[j] = sum_i dZ[i][j] in two passes with a fixed order: CTA (cx, r) sums
// its row slice of columns 32 cx .. 32 cx + 31 (thread (x, y): rows y, y + 8,
// ... of the slice, then a tree over y) into part[r][j]; then the slices are
// added in order.  FP32 sums of at most a few thousand rows.
constexpr int kColSlices = 16;

__global__ void colsum_partial_kernel(int64_t M, int N, const float *dZ, float *part)
{
    __shared__ float red[8][33];
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + x;
    const int64_t per = (M + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = blockIdx.y * per, r1 = min(M, r0 + per);
    float acc = 0.f;
    if (j < N)
        for (int64_t i = r0 + y; i < r1; i += 8) acc += dZ[i * N + j];
    red[y][x] = acc;
    __syncthreads();
    for (int st = 4; st > 0; st >>= 1) {
        if (y < st) red[y][x] += red[y + st][x];
        __syncthreads();
    }
    if (y == 0 && j < N) part[(int64_t)blockIdx.y * N + j] = red[0][x];
}

__global__ void colsum_final_kernel(int N, int slices, const float *part, float *db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int r = 0; r < slices; ++r) s += part[(int64_t)r * N + j];
    db[j] = s;
}

__global__ void adam_kernel(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Normalised stencil features of nodes idx[0..k) (all nodes when idx == null).
__global__ void features_kernel(int Nx, int Ny, int Nz, int64_t base, int64_t k,
                                const int32_t *idx,
                                const double *Vn, const double *y, const double *d1,
                                const double *d2, const float *mean, const float *stdv, float *X)
{
    const int nx = Nx + 1, ny = Ny + 1, nz = Nz + 1;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < k;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int node = idx ? idx[r] : (int)(base + r);
        const int i = node % nx, j = (node / nx) % ny, kk = node / (nx * ny);
        float *x = X + r * NI;
        int s = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++s) {
                    const int ii = i + dx, jj = j + dy, kz = kk + dz;
                    const bool ok = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kz >= 0 && kz < nz;
                    const int nb = ok ? ii + nx * (jj + ny * kz) : 0;
                    for (int c = 0; c < 4; ++c) {
                        const double raw = ok ? (c < 3 ? Vn[4 * (int64_t)nb + c]
                                                       : y[4 * (int64_t)nb + 3])
                                              : 0.0;
                        const int f = 4 * s + c;
                        x[f] = (float)((raw - mean[f]) / stdv[f]);
                    }
                }
        for (int c = 0; c < 4; ++c) {
            const int f = 108 + c;
            const double e = 2.0 * d1[4 * (int64_t)node + c] - d2[4 * (int64_t)node + c];
            x[f] = (float)((e - mean[f]) / stdv[f]);
        }
    }
}

// y0 = y + e + (mean_c + std_c * O) for nodes [base, base + k)
__global__ void predict_combine_kernel(int64_t base, int64_t k, const double *y, const double *d1,
                                       const double *d2, const float *O, const float *omean,
                                       const float *ostd, double *y0)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < k;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = base + r;
        for (int c = 0; c < 4; ++c) {
            const int64_t q = 4 * node + c;
            const double e = 2.0 * d1[q] - d2[q];
            y0[q] = y[q] + e + ((double)omean[c] + (double)ostd[c] * (double)O[r * NO + c]);
        }
    }
}

// fallback predictors: mode 0 y0 = y (zero increment), mode 1 y0 = y + e
__global__ void fallback_kernel(int64_t n4, int mode, const double *y, const double *d1,
                                const double *d2, double *y0)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
         q += (int64_t)gridDim.x * blockDim.x)
        y0[q] = mode == 1 ? y[q] + 2.0 * d1[q] - d2[q] : y[q];
}

__global__ void apply_dirichlet_kernel(int64_t n4, const uint8_t *mask, const double *yD,
                                       double *y)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
         q += (int64_t)gridDim.x * blockDim.x)
        if (mask[q]) y[q] = yD[q];
}

// One search direction of the fitted predictor, in FP32 (which: 0 the last
// increment d1; 1 the one before, d2; 2 the network's correction
// c = ml - yn - (2 d1 - d2)); zero on Dirichlet rows
constexpr int kFitDirs = 3;
__global__ void direction_kernel(int64_t n4, int which, const double *ml, const double *yn,
                                 const double *d1, const double *d2, const uint8_t *mask,
                                 float *out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (which == 0)
            v = d1[q];
        else if (which == 1)
            v = d2[q];
        else
            v = ml[q] - yn[q] - (2.0 * d1[q] - d2[q]);
        if (mask && mask[q]) v = 0.0;
        out[q] = (float)v;
    }
}

// y = yfb + x0 d1 + x1 d2 + x2 c (Dirichlet rows = yD)
__global__ void fitted_kernel(int64_t n4, const double *yfb, const double *ml, const double *yn,
                              const double *d1, const double *d2, const uint8_t *mask,
                              const double *yD, double x0, double x1, double x2, double *y)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double corr = ml[q] - yn[q] - (2.0 * d1[q] - d2[q]);
        y[q] = (mask && mask[q]) ? yD[q] : yfb[q] + x0 * d1[q] + x1 * d2[q] + x2 * corr;
    }
}

// The fit's sums on the FP32 pipe: each product is split exactly (TwoProd:
// p = x y rounded, e = fma(x, y, -p)) and added into a compensated pair
// (s, c) (TwoSum of s and p, the errors gathered in c), about 2^-44 relative
// per thread's sum; the CTA sums the pairs in FP64.  The residual's doubles
// enter truncated to float (2^-23 relative per entry; the fit is a
// least-squares model of three coefficients, judged afterwards by the true
// residual of its candidate), formed from their bits by integer operations.
// (FP64 products and sums took 555 us at 128^3: GB300's FP64 unit issues two
// operations per SM and clock, and a double -> float conversion is one.)
struct FitAcc {
    float s, c;
};
__device__ __forceinline__ void fit_add(FitAcc &a, float p, float e)
{
    const float s = __fadd_rn(a.s, p);
    const float bb = __fsub_rn(s, a.s);
    const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(e, t));
}
// a += x y
__device__ __forceinline__ void fit_mul(FitAcc &a, float x, float y)
{
    const float p = __fmul_rn(x, y);
    fit_add(a, p, __fmaf_rn(x, y, -p));
}
// the float of a double with its significand truncated to 24 bits, from the
// bits (no FP64 operation): zero below the float range, infinite above it,
// NaN stays NaN
__device__ __forceinline__ float trunc_to_float(double r)
{
    const long long b = __double_as_longlong(r);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ff);
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (mant | ((b & 0xfffffffffffffLL) != 0)));
    const int fe = e - 1023 + 127;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)fe << 23) | mant);
}

// per-block partial sums (FP64) of kSums compensated pairs in red
template <int kSums, int kThreads>
__device__ __forceinline__ void fit_block_sums(const FitAcc (&acc)[kSums], double (*red)[kThreads],
                                               double *partial)
{
#pragma unroll
    for (int k = 0; k < kSums; ++k) red[k][threadIdx.x] = (double)acc[k].s + (double)acc[k].c;
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int k = 0; k < kSums; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < kSums) partial[kSums * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// per-block partial sums of the normal equations of the fit: G_ij = J_i . J_j
// (i <= j, 6 values, row by row), r_i = J_i . R (3 values) and |R|^2 (the
// model's; the fallback's reported norm is within 1e-6 of the FP64 one)
constexpr int kFitBlocks = 608, kFitThreads = 256;  // 4 per SM of a GB300
// doubles of per-block partial sums the handle keeps (the fit's 10 per block,
// the training loss's one per block)
constexpr int kPartialDoubles = 8192;
static_assert((kFitDirs * (kFitDirs + 1) / 2 + kFitDirs + 1) * kFitBlocks <= kPartialDoubles,
              "partial sums of the fit");
constexpr int kFitSums = kFitDirs * (kFitDirs + 1) / 2 + kFitDirs;
__global__ void __launch_bounds__(kFitThreads) fit_dots_kernel(int64_t n4, const float *Jd,
                                                               const double *R, double *partial)
{
    __shared__ double red[kFitSums + 1][kFitThreads];
    FitAcc acc[kFitSums + 1];
#pragma unroll
    for (int k = 0; k <= kFitSums; ++k) acc[k] = {0.0f, 0.0f};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float a[kFitDirs];
#pragma unroll
        for (int d = 0; d < kFitDirs; ++d) a[d] = Jd[d * n4 + i];
        const float r = trunc_to_float(R[i]);
        int k = 0;
#pragma unroll
        for (int d = 0; d < kFitDirs; ++d)
#pragma unroll
            for (int e = d; e < kFitDirs; ++e) fit_mul(acc[k++], a[d], a[e]);
#pragma unroll
        for (int d = 0; d < kFitDirs; ++d) fit_mul(acc[k++], a[d], r);
        fit_mul(acc[k], r, r);
    }
    fit_block_sums<kFitSums + 1, kFitThreads>(acc, red, partial);
}

// per-block partial sums of |x|^2 in FP64 (the reported norm of a judged
// residual: to FP64 accuracy), on a grid that keeps the FP64 unit busy
__global__ void __launch_bounds__(kFitThreads) sumsq_kernel(int64_t n, const double *x,
                                                            double *partial)
{
    __shared__ double red[kFitThreads];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(x[i], x[i], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = kFitThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

int blocks(int64_t n, int threads = 256, int cap = sm_count() * 16)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// db = column sums of dZ [M][N] (the bias gradient), through the split-K
// workspace (free between GEMMs in stream order)
fsi_status colsum(const fsi_mlp *h, int64_t M, int N, const float *dZ, float *db)
{
    dim3 grid((N + 31) / 32, kColSlices);
    colsum_partial_kernel<<<grid, 256, 0, h->stream>>>(M, N, dZ, h->gemm_work);
    colsum_final_kernel<<<(N + 255) / 256, 256, 0, h->stream>>>(N, kColSlices, h->gemm_work, db);
    return check_launch("bias gradient");
}

fsi_status forward_impl(fsi_mlp *h, const float *P, const float *X, int64_t B, bool keep)
{
    FSI_TRY(gemm(h, ga((int)B, NH, NI, X, NI, 0, P + OFF_W1, NH, 0, h->H1, NH, EPI_BIAS_RELU,
                       P + OFF_b1, keep ? h->Z1 : nullptr)));
    FSI_TRY(gemm(h, ga((int)B, NH, NH, h->H1, NH, 0, P + OFF_W2, NH, 0, h->H2, NH, EPI_BIAS_RELU,
                       P + OFF_b2, keep ? h->Z2 : nullptr)));
    return gemm(h, ga((int)B, NO, NH, h->H2, NH, 0, P + OFF_W3, NO, 0, h->O, NO, EPI_BIAS,
                      P + OFF_b3));
}

// the tensor-core kernels' wait-timeout flag, read (after the caller's
// synchronisation) and cleared
fsi_status take_tc_error(fsi_mlp *h)
{
    int f = 0;
    FSI_CUDA(cudaMemcpy(&f, h->tc_err, sizeof f, cudaMemcpyDeviceToHost), "memcpy");
    if (!f) return FSI_OK;
    FSI_CUDA(cudaMemset(h->tc_err, 0, sizeof(int)), "memset");
    return set_error(FSI_ERR_TIMEOUT, "a tensor-core wait ran out (network kernels)");
}

fsi_status check_mlp(const fsi_mlp *h, int64_t B)
{
    if (!h) return set_error(FSI_ERR_ARG, "mlp handle is NULL");
    if (B < 1 || B > h->max_batch)
        return set_error(FSI_ERR_ARG, "batch %lld outside [1, %lld]", (long long)B,
                         (long long)h->max_batch);
    return FSI_OK;
}

}  // namespace
}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status fsi_mlp_create(int device, void *cuda_stream, int64_t max_batch, fsi_mlp **out)
{
    if (!out) return set_error(FSI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 24))
        return set_error(FSI_ERR_ARG, "max_batch must be in [1, 2^24]");
    FSI_DEVICE(device);
    fsi_mlp *h = new (std::nothrow) fsi_mlp();
    if (!h) return set_error(FSI_ERR_OOM, "host allocation failed");
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    h->max_batch = max_batch;
    struct {
        float **p;
        int64_t n;
    } req[] = {{&h->Z1, NH}, {&h->H1, NH}, {&h->Z2, NH}, {&h->H2, NH}, {&h->O, NO},
               {&h->dO, NO}, {&h->dZ1, NH}, {&h->dZ2, NH}, {&h->X, NI}};
    for (auto &r : req) {
        cudaError_t e = cudaMalloc(r.p, (size_t)max_batch * r.n * sizeof(float));
        if (e != cudaSuccess) {
            fsi_mlp_destroy(h);
            return check_cuda(e, "mlp activation allocation");
        }
    }
    cudaError_t e = cudaMalloc(&h->loss_partial, kPartialDoubles * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->packed, mlp_tc_packed_bytes());
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->gemm_work, tc_gemm_work_floats() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(h->tc_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        fsi_mlp_destroy(h);
        return check_cuda(e, "mlp allocation");
    }
    *out = h;
    return FSI_OK;
}

void fsi_mlp_destroy(fsi_mlp *h)
{
    if (!h) return;
    fsi::DeviceGuard _fsi_device_guard(h->device);
    cudaStreamSynchronize(h->stream);
    float *ptrs[] = {h->Z1, h->H1, h->Z2, h->H2, h->O, h->dO, h->dZ1, h->dZ2, h->X};
    for (float *p : ptrs) cudaFree(p);
    cudaFree(h->loss_partial);
    cudaFree(h->packed);
    cudaFree(h->tc_err);
    cudaFree(h->gemm_work);
    delete h;
}

int64_t fsi_mlp_num_params(void) { return N_PARAMS; }

fsi_status fsi_mlp_forward(fsi_mlp *h, const float *params, const float *X, int64_t B, float *out)
{
    FSI_TRY(check_mlp(h, B));
    if (!params || !X || !out) return set_error(FSI_ERR_ARG, "NULL argument");
    FSI_DEVICE(h->device);
    FSI_TRY(forward_impl(h, params, X, B, false));
    FSI_CUDA(cudaMemcpyAsync(out, h->O, B * NO * sizeof(float), cudaMemcpyDeviceToDevice,
                             h->stream),
             "memcpy");
    return FSI_OK;
}

fsi_status fsi_mlp_loss_grad(fsi_mlp *h, const float *params, const float *X, const float *T,
                             int64_t B, float *loss, float *grad)
{
    FSI_TRY(check_mlp(h, B));
    if (!params || !X || !T || !loss || !grad) return set_error(FSI_ERR_ARG, "NULL argument");
    FSI_DEVICE(h->device);
    cudaStream_t s = h->stream;
    const float *P = params;
    FSI_TRY(forward_impl(h, P, X, B, true));
    const int nb = 256;
    loss_kernel<<<nb, 256, 0, s>>>(B, h->O, T, h->dO, h->loss_partial);
    loss_final_kernel<<<1, 32, 0, s>>>(nb, h->loss_partial, loss);
    FSI_TRY(check_launch("loss kernels"));
    const int M = (int)B;
    // layer 3: dW3 = H2^T dO, db3 = colsum(dO), dZ2 = (dO W3^T) * (Z2 > 0)
    FSI_TRY(gemm(h, ga(NH, NO, M, h->H2, NH, 1, h->dO, NO, 0, grad + OFF_W3, NO)));
    FSI_TRY(colsum(h, B, NO, h->dO, grad + OFF_b3));
    FSI_TRY(gemm(h, ga(M, NH, NO, h->dO, NO, 0, P + OFF_W3, NO, 1, h->dZ2, NH, EPI_MASK,
                       nullptr, nullptr, h->Z2)));
    // layer 2: dW2 = H1^T dZ2, db2, dZ1 = (dZ2 W2^T) * (Z1 > 0)
    FSI_TRY(gemm(h, ga(NH, NH, M, h->H1, NH, 1, h->dZ2, NH, 0, grad + OFF_W2, NH)));
    FSI_TRY(colsum(h, B, NH, h->dZ2, grad + OFF_b2));
    FSI_TRY(gemm(h, ga(M, NH, NH, h->dZ2, NH, 0, P + OFF_W2, NH, 1, h->dZ1, NH, EPI_MASK,
                       nullptr, nullptr, h->Z1)));
    // layer 1: dW1 = X^T dZ1, db1
    FSI_TRY(gemm(h, ga(NI, NH, M, X, NI, 1, h->dZ1, NH, 0, grad + OFF_W1, NH)));
    return colsum(h, B, NH, h->dZ1, grad + OFF_b1);
}

fsi_status fsi_mlp_adam(fsi_mlp *h, float *params, const float *grad, float *m, float *v,
                        int step, float lr, float beta1, float beta2, float eps)
{
    if (!h) return set_error(FSI_ERR_ARG, "mlp handle is NULL");
    if (!params || !grad || !m || !v || step < 1) return set_error(FSI_ERR_ARG, "bad argument");
    FSI_DEVICE(h->device);
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<blocks(N_PARAMS), 256, 0, h->stream>>>(N_PARAMS, params, grad, m, v, lr, beta1,
                                                        beta2, eps, c1, c2);
    return check_launch("adam kernel");
}

fsi_status fsi_mlp_features(fsi_mesh *mesh, const double *Vn, const double *y, const double *d1,
                            const double *d2, const int32_t *idx, int64_t k,
                            const float *in_mean, const float *in_std, float *X)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(require_structured(mesh, "fsi_mlp_features (3x3x3 stencil features)"));
    if (!Vn || !y || !d1 || !d2 || !in_mean || !in_std || !X)
        return set_error(FSI_ERR_ARG, "NULL argument");
    if (!idx) k = mesh->n_nodes;
    if (k < 0) return set_error(FSI_ERR_ARG, "k < 0");
    if (k == 0) return FSI_OK;
    FSI_DEVICE(mesh->device);
    features_kernel<<<blocks(k), 256, 0, mesh->stream>>>(mesh->grid.N[0], mesh->grid.N[1],
                                                        mesh->grid.N[2], 0, k, idx, Vn, y, d1,
                                                        d2, in_mean, in_std, X);
    return check_launch("features kernel");
}

fsi_status fsi_mlp_predict(fsi_mlp *h, fsi_mesh *mesh, const float *params, const float *in_mean,
                           const float *in_std, const float *out_mean, const float *out_std,
                           const double *Vn, const double *y, const double *d1, const double *d2,
                           double *y0)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(require_structured(mesh, "fsi_mlp_predict (3x3x3 stencil features)"));
    if (!h) return set_error(FSI_ERR_ARG, "mlp handle is NULL");
    if (!params || !in_mean || !in_std || !out_mean || !out_std || !Vn || !y || !d1 || !d2 || !y0)
        return set_error(FSI_ERR_ARG, "NULL argument");
    if (h->device != mesh->device) return set_error(FSI_ERR_ARG, "mlp and mesh on other devices");
    FSI_DEVICE(mesh->device);
    // fused features -> network -> predictor on the tcgen05 tensor cores
    return mlp_predict_tc(mesh->stream, mesh->device, mesh->grid, mesh->n_nodes, params, in_mean,
                          in_std, out_mean, out_std, Vn, y, d1, d2, y0, h->packed, h->tc_err);
}

fsi_status fsi_mlp_guess(fsi_mlp *h, fsi_mesh *mesh, const float *params, const float *in_mean,
                         const float *in_std, const float *out_mean, const float *out_std,
                         const fsi_step_state *st, const double *yn, const double *d1,
                         const double *d2, int fallback, fsi_prec judge_prec, double *work,
                         fsi_guess_report *rep)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(require_structured(mesh, "fsi_mlp_guess (3x3x3 stencil features)"));
    if (!h || !st || !st->y || !yn || !d1 || !d2 || !work || !rep)
        return set_error(FSI_ERR_ARG, "NULL argument");
    if (fallback != 0 && fallback != 1) return set_error(FSI_ERR_ARG, "fallback must be 0 or 1");
    if (judge_prec != FSI_F64 && judge_prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "judge_prec must be FSI_F64 or FSI_DF64");
    if (st->y == yn) return set_error(FSI_ERR_ARG, "st->y must not alias yn");
    FSI_TRY(validate_step_state(mesh, st));
    FSI_DEVICE(mesh->device);
    cudaStream_t s = mesh->stream;
    const int64_t n4 = 4 * mesh->n_nodes;
    // work: [0] the network's predictor, [1] R(y_fb), [2..4] FP32: the three
    // directions and their J d_i; once the fit is done [2] holds the fitted
    // candidate and [3] its residual
    double *ml = work, *Rfb = work + n4, *cand = work + 2 * n4, *Rc = work + 3 * n4;
    float *dir = (float *)(work + 2 * n4), *Jd = dir + kFitDirs * n4;
    // the fallback predictor (in st->y) and the network's predictor (in ml)
    fallback_kernel<<<blocks(n4), 256, 0, s>>>(n4, fallback, yn, d1, d2, st->y);
    FSI_TRY(check_launch("fallback kernel"));
    FSI_TRY(fsi_mlp_predict(h, mesh, params, in_mean, in_std, out_mean, out_std, st->Vn, yn, d1,
                            d2, ml));
    if (st->mask) {
        apply_dirichlet_kernel<<<blocks(n4), 256, 0, s>>>(n4, st->mask, st->yD, st->y);
        FSI_TRY(check_launch("dirichlet kernel"));
    }
    // one FP32 linearisation at y_fb: the fallback's residual for the fit
    // (its VMS part in FP32: the fit needs it to far less than the 1e-3 of
    // ||R|| that a predictor gains; coupling and Dirichlet rows double-float)
    // and J applied to d1, d2, c
    for (int i = 0; i < kFitDirs; ++i)
        direction_kernel<<<blocks(n4), 256, 0, s>>>(n4, i, ml, yn, d1, d2, st->mask, dir + i * n4);
    FSI_TRY(check_launch("direction kernel"));
    {
        const float *xs[kFitDirs];
        float *js[kFitDirs];
        for (int i = 0; i < kFitDirs; ++i) {
            xs[i] = dir + i * n4;
            js[i] = Jd + i * n4;
        }
        FSI_TRY(coupled_jacobian_f32(mesh, st, kFitDirs, xs, js, Rfb));
    }
    // normal equations G x = -r of min |R_fb + sum_i x_i J d_i|
    fit_dots_kernel<<<kFitBlocks, kFitThreads, 0, s>>>(n4, Jd, Rfb, h->loss_partial);
    FSI_TRY(check_launch("fit dots"));
    std::vector<double> hp((kFitSums + 1) * kFitBlocks);
    FSI_CUDA(cudaMemcpyAsync(hp.data(), h->loss_partial, hp.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, s),
             "memcpy");
    FSI_CUDA(cudaStreamSynchronize(s), "sync");
    double q[kFitSums] = {}, rr = 0.0;
    for (int b = 0; b < kFitBlocks; ++b) {
        for (int k = 0; k < kFitSums; ++k) q[k] += hp[(kFitSums + 1) * b + k];
        rr += hp[(kFitSums + 1) * b + kFitSums];
    }
    const double r_fb = std::sqrt(rr);
    constexpr int K = kFitDirs;
    double G[K][K], r[K];
    {
        int k = 0;
        for (int i = 0; i < K; ++i)
            for (int j = i; j < K; ++j) G[i][j] = G[j][i] = q[k++];
        for (int i = 0; i < K; ++i) r[i] = q[k++];
    }
    // min over the directions in `sel` (a bit mask) of the linear model
    // |R_fb + sum x_i J d_i|^2: Cholesky with pivot tolerance (a direction
    // whose Schur pivot is below 1e-12 of its own norm adds nothing and keeps
    // coefficient 0); returns the model's |R|^2
    auto fit = [&](unsigned sel, double (&x)[K]) {
        bool use[K];
        double L[K][K] = {};
        for (int i = 0; i < K; ++i) {
            double d = G[i][i];
            for (int k = 0; k < i; ++k) d -= L[i][k] * L[i][k];
            use[i] = ((sel >> i) & 1u) && G[i][i] > 0.0 && d > 1e-12 * G[i][i];
            L[i][i] = use[i] ? std::sqrt(d) : 0.0;
            for (int j = i + 1; j < K; ++j) {
                double t = G[j][i];
                for (int k = 0; k < i; ++k) t -= L[j][k] * L[i][k];
                L[j][i] = use[i] ? t / L[i][i] : 0.0;
            }
        }
        double z[K];
        for (int i = 0; i < K; ++i) {
            double t = -r[i];
            for (int k = 0; k < i; ++k) t -= L[i][k] * z[k];
            z[i] = use[i] ? t / L[i][i] : 0.0;
        }
        for (int i = K - 1; i >= 0; --i) {
            double t = z[i];
            for (int k = i + 1; k < K; ++k) t -= L[k][i] * x[k];
            x[i] = use[i] ? t / L[i][i] : 0.0;
        }
        double v = rr;
        for (int i = 0; i < K; ++i) {
            v += 2.0 * x[i] * r[i];
            for (int j = 0; j < K; ++j) v += x[i] * G[i][j] * x[j];
        }
        return std::max(v, 0.0);
    };
    double x[K];
    fit(0x7u, x);
    // the same model over the history directions alone (the fit without the
    // network), and at the network's own predictor y_n + e + c (e = 2 d1 - d2)
    {
        double xh[K];
        rep->r_history_fit = std::sqrt(fit(0x3u, xh));
        const double xm[K] = {fallback == 1 ? 0.0 : 2.0, fallback == 1 ? 0.0 : -1.0, 1.0};
        double v = rr;
        for (int i = 0; i < K; ++i) {
            v += 2.0 * xm[i] * r[i];
            for (int j = 0; j < K; ++j) v += xm[i] * G[i][j] * xm[j];
        }
        rep->r_learned = std::sqrt(std::max(v, 0.0));
    }
    rep->r_fallback = r_fb;
    rep->c_d1 = x[0];
    rep->c_d2 = x[1];
    rep->c_net = x[2];
    // the candidate, judged by its own residual in judge_prec
    fitted_kernel<<<blocks(n4), 256, 0, s>>>(n4, st->y, ml, yn, d1, d2, st->mask, st->yD, x[0],
                                            x[1], x[2], cand);
    FSI_TRY(check_launch("fitted kernel"));
    fsi_step_state tmp = *st;
    tmp.y = cand;
    FSI_TRY(fsi_coupled_residual(mesh, judge_prec, &tmp, Rc));
    sumsq_kernel<<<kFitBlocks, kFitThreads, 0, s>>>(n4, Rc, h->loss_partial);
    FSI_TRY(check_launch("norm kernel"));
    std::vector<double> hn(kFitBlocks);
    FSI_CUDA(cudaMemcpyAsync(hn.data(), h->loss_partial, hn.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, s),
             "memcpy");
    FSI_CUDA(cudaStreamSynchronize(s), "sync");
    double rc = 0.0;
    for (int b = 0; b < kFitBlocks; ++b) rc += hn[b];
    rep->r_combined = std::sqrt(rc);
    rep->used = std::isfinite(rep->r_combined) && rep->r_combined < r_fb ? 2 : 0;
    if (rep->used == 2)
        FSI_CUDA(cudaMemcpyAsync(st->y, cand, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s),
                 "memcpy");
    // the judged residual of the returned predictor, for the Newton step (the
    // fallback's in judge_prec when it is kept)
    if (rep->used == 2)
        FSI_CUDA(cudaMemcpyAsync(work, Rc, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s),
                 "memcpy");
    else
        FSI_TRY(fsi_coupled_residual(mesh, judge_prec, st, work));
    FSI_CUDA(cudaStreamSynchronize(s), "sync");
    return take_tc_error(h);
}

fsi_status fsi_mlp_check(fsi_mlp *h)
{
    if (!h) return set_error(FSI_ERR_ARG, "mlp handle is NULL");
    FSI_DEVICE(h->device);
    FSI_CUDA(cudaDeviceSynchronize(), "device sync");
    return take_tc_error(h);
}

}  // extern "C"
