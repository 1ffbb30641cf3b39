// runtime.cu -- handles, errors, validation and the generalized-alpha stage
// kernel of libfsi (C ABI in include/fsi.h).
#include <atomic>
#include <mutex>
#include <set>
#include <tuple>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fsi_internal.cuh"

namespace fsi {

static thread_local std::string g_last_error;

fsi_status set_error(fsi_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

fsi_status check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return FSI_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(FSI_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(FSI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

fsi_status check_launch(const char *what) { return check_cuda(cudaGetLastError(), what); }

DeviceGuard::DeviceGuard(int device)
{
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != device) st_ = check_cuda(cudaSetDevice(device), "cudaSetDevice");
}

DeviceGuard::~DeviceGuard()
{
    int cur = -1;
    if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
}

fsi_status set_smem_limit(const void *kernel, int bytes)
{
    static std::mutex mu;
    static std::set<std::tuple<const void *, int, int>> done;
    int dev = 0;
    FSI_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(kernel, dev, bytes);
    if (done.count(key)) return FSI_OK;
    FSI_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
             "cudaFuncSetAttribute");
    done.insert(key);
    return FSI_OK;
}

int sm_count()
{
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cached[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
    if (dev < kMaxDevices) {
        int v = cached[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 152;
    if (dev < kMaxDevices) cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

static fsi_status validate_physics(const fsi_physics *p)
{
    if (!p) return set_error(FSI_ERR_ARG, "physics is NULL");
    if (!(p->rho > 0.0) || !(p->mu >= 0.0) || !(p->dt > 0.0) || !(p->C_I >= 0.0) ||
        !(p->C_T >= 0.0) || !(p->rho_inf >= 0.0 && p->rho_inf <= 1.0) ||
        !std::isfinite(p->rho) || !std::isfinite(p->mu) || !std::isfinite(p->dt))
        return set_error(FSI_ERR_ARG,
                         "invalid physics: need rho > 0, mu >= 0, dt > 0, C_I, C_T >= 0, "
                         "0 <= rho_inf <= 1");
    return FSI_OK;
}

static void derive(fsi_mesh *m)
{
    const double r = m->phys.rho_inf;
    m->alpha_m = 0.5 * (3.0 - r) / (1.0 + r);
    m->alpha_f = 1.0 / (1.0 + r);
    m->gamma = 0.5 + m->alpha_m - m->alpha_f;
}

fsi_status validate_mesh(const fsi_mesh *m)
{
    if (!m) return set_error(FSI_ERR_ARG, "mesh is NULL");
    return FSI_OK;
}

fsi_status require_structured(const fsi_mesh *m, const char *what)
{
    if (m->tet) return set_error(FSI_ERR_ARG, "%s needs a structured grid (not a tetrahedral mesh)",
                                 what);
    return FSI_OK;
}

size_t vms_scratch_bytes_for(const fsi_mesh *m, const Brick &b, size_t elem_bytes)
{
    const int *N = m->grid.N;
    size_t nb = (size_t)((N[0] + b.bx - 1) / b.bx) * ((N[1] + b.by - 1) / b.by) *
                ((N[2] + b.bz - 1) / b.bz);
    size_t nodes = (size_t)(b.bx + 1) * (b.by + 1) * (b.bz + 1);
    return nb * nodes * 4 * elem_bytes;
}

fsi_status ensure_vms_scratch(fsi_mesh *m, const Brick &b, size_t elem_bytes)
{
    size_t need = vms_scratch_bytes_for(m, b, elem_bytes);
    if (need <= m->vms_scratch_bytes) return FSI_OK;
    if (m->vms_scratch) {
        FSI_CUDA(cudaStreamSynchronize(m->stream), "stream sync before scratch growth");
        cudaFree(m->vms_scratch);
        m->vms_scratch = nullptr;
        m->vms_scratch_bytes = 0;
    }
    FSI_CUDA(cudaMalloc(&m->vms_scratch, need), "VMS scratch allocation");
    m->vms_scratch_bytes = need;
    return FSI_OK;
}

fsi_status ensure_spread_scratch(fsi_mesh *m, size_t need)
{
    if (need <= m->spread_scratch_bytes) return FSI_OK;
    if (m->spread_scratch) {
        FSI_CUDA(cudaStreamSynchronize(m->stream), "stream sync before scratch growth");
        cudaFree(m->spread_scratch);
        m->spread_scratch = nullptr;
        m->spread_scratch_bytes = 0;
    }
    FSI_CUDA(cudaMalloc(&m->spread_scratch, need), "spread scratch allocation");
    m->spread_scratch_bytes = need;
    return FSI_OK;
}

// ------------------------------------------------------------ stage kernel
template <typename T>
__global__ void stage_kernel(int64_t n, T dt, T am, T af, T gamma, const vec4<T> *__restrict__ y,
                             const vec4<T> *__restrict__ Vn, const vec4<T> *__restrict__ An,
                             const T *__restrict__ s, vec4<T> *__restrict__ U,
                             vec4<T> *__restrict__ A)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vec4<T> yy = ld4(y + i), v = ld4(Vn + i), a = ld4(An + i);
        // V_{n+1} = V_n + dt Vdot_n + gamma dt (Vdot_{n+1} - Vdot_n)
        T v1x = v.x + dt * a.x + gamma * dt * (yy.x - a.x);
        T v1y = v.y + dt * a.y + gamma * dt * (yy.y - a.y);
        T v1z = v.z + dt * a.z + gamma * dt * (yy.z - a.z);
        vec4<T> u, acc;
        u.x = v.x + af * (v1x - v.x);
        u.y = v.y + af * (v1y - v.y);
        u.z = v.z + af * (v1z - v.z);
        u.w = yy.w;
        acc.x = a.x + am * (yy.x - a.x);
        acc.y = a.y + am * (yy.y - a.y);
        acc.z = a.z + am * (yy.z - a.z);
        acc.w = s ? s[i] : T(1);
        U[i] = u;
        A[i] = acc;
    }
}

// V_n <- V_{n+1} = V_n + dt Vdot_n + gamma dt (Vdot_{n+1} - Vdot_n), Vdot_n <- Vdot_{n+1}
template <typename T>
__global__ void advance_kernel(int64_t n, T dt, T gamma, const vec4<T> *__restrict__ y,
                               vec4<T> *__restrict__ Vn, vec4<T> *__restrict__ An)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vec4<T> yy = ld4(y + i), v = Vn[i], a = An[i];
        v.x = v.x + dt * a.x + gamma * dt * (yy.x - a.x);
        v.y = v.y + dt * a.y + gamma * dt * (yy.y - a.y);
        v.z = v.z + dt * a.z + gamma * dt * (yy.z - a.z);
        a.x = yy.x;
        a.y = yy.y;
        a.z = yy.z;
        Vn[i] = v;
        An[i] = a;
    }
}

static int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    const int cap = sm_count() * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace fsi

using namespace fsi;

extern "C" {

const char *fsi_last_error(void) { return g_last_error.c_str(); }

fsi_status fsi_mesh_create(const fsi_grid *grid, const fsi_physics *phys, int device,
                           void *cuda_stream, fsi_mesh **out)
{
    if (!out) return set_error(FSI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid) return set_error(FSI_ERR_ARG, "grid is NULL");
    FSI_TRY(validate_physics(phys));
    int64_t n = 1, E = 1;
    for (int k = 0; k < 3; ++k) {
        if (grid->N[k] < 1 || !(grid->h[k] > 0.0) || !std::isfinite(grid->h[k]) ||
            !std::isfinite(grid->x0[k]))
            return set_error(FSI_ERR_ARG, "invalid grid: need N[k] >= 1 and finite h[k] > 0");
        n *= (int64_t)grid->N[k] + 1;
        E *= grid->N[k];
    }
    if (n > INT32_MAX) return set_error(FSI_ERR_ARG, "grid has more than 2^31-1 nodes");
    int ndev = 0;
    FSI_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev)
        return set_error(FSI_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
    FSI_DEVICE(device);
    fsi_mesh *m = new (std::nothrow) fsi_mesh();
    if (!m) return set_error(FSI_ERR_OOM, "host allocation of the mesh handle failed");
    m->grid = *grid;
    m->phys = *phys;
    m->device = device;
    m->stream = (cudaStream_t)cuda_stream;
    m->n_nodes = n;
    m->n_elems = E;
    derive(m);
    // the fused pass keeps two element buffers in shared memory: half as many
    // elements per brick keeps two CTAs per SM
    for (int op = 0; op < 3; ++op)
        for (int p = 0; p < 3; ++p)
            m->brick[op][p] = op == 2 ? Brick{8, 4, 4, 256} : Brick{8, 8, 4, 256};
    fsi_status st = FSI_OK;
    // cell-hash scratch: fill counters [E+1], scan scratch, counters; both
    // start at zero and every cell-table build leaves them so
    int64_t nblk = cell_table_scan_ints(E);
    m->scan_tmp_len = nblk;
    if (st == FSI_OK)
        st = check_cuda(cudaMalloc(&m->hash_fill, (E + 1) * sizeof(int32_t)), "hash scratch");
    if (st == FSI_OK)
        st = check_cuda(cudaMalloc(&m->scan_tmp, nblk * sizeof(int32_t)), "scan scratch");
    if (st == FSI_OK)
        st = check_cuda(cudaMemset(m->hash_fill, 0, (E + 1) * sizeof(int32_t)), "hash scratch");
    if (st == FSI_OK)
        st = check_cuda(cudaMemset(m->scan_tmp, 0, nblk * sizeof(int32_t)), "scan scratch");
    m->hash_clean = st == FSI_OK;
    if (st == FSI_OK)
        st = check_cuda(cudaMalloc(&m->dev_counters, 8 * sizeof(int64_t)), "counter scratch");
    if (st == FSI_OK) st = ensure_vms_scratch(m, m->brick[1][0], sizeof(double));
    if (st == FSI_OK) st = ensure_spread_scratch(m, (size_t)E * 24 * sizeof(double));
    if (st != FSI_OK) {
        fsi_mesh_destroy(m);
        return st;
    }
    *out = m;
    return FSI_OK;
}

void fsi_mesh_destroy(fsi_mesh *m)
{
    if (!m) return;
    fsi::DeviceGuard _fsi_device_guard(m->device);
    cudaStreamSynchronize(m->stream);
    cudaFree(m->vms_scratch);
    cudaFree(m->hash_fill);
    cudaFree(m->scan_tmp);
    cudaFree(m->pt_tmp);
    cudaFree(m->dev_counters);
    cudaFree(m->spread_scratch);
    destroy_newton_workspace(m);
    destroy_pmg(m);
    destroy_amg(m);
    cudaFree(m->coords64);
    cudaFree(m->coords32);
    for (void *g : m->map_geo) cudaFree(g);
    if (m->tet) fsi_tetmesh_destroy(m->tet);
    delete m;
}

fsi_status fsi_mesh_set_stream(fsi_mesh *m, void *cuda_stream)
{
    FSI_TRY(validate_mesh(m));
    m->stream = (cudaStream_t)cuda_stream;
    if (m->tet) tet_set_stream(m->tet, m->stream);
    return FSI_OK;
}

namespace {
__global__ void pad_coords_kernel(int64_t n, const double *X, double4 *C64, float4 *C32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
        C64[i] = make_double4(x, y, z, 0.0);
        C32[i] = make_float4((float)x, (float)y, (float)z, 0.0f);
    }
}
}  // namespace

fsi_status fsi_mesh_set_coordinates(fsi_mesh *m, const double *X)
{
    FSI_TRY(validate_mesh(m));
    FSI_TRY(require_structured(m, "fsi_mesh_set_coordinates"));
    FSI_DEVICE(m->device);
    FSI_CUDA(cudaStreamSynchronize(m->stream), "sync");
    for (void *&g : m->map_geo) {
        cudaFree(g);
        g = nullptr;
    }
    destroy_amg(m);  // assembled from the old coordinates
    if (!X) {
        cudaFree(m->coords64);
        cudaFree(m->coords32);
        m->coords64 = m->coords32 = nullptr;
        return FSI_OK;
    }
    if (!m->coords64) {
        if (cudaMalloc(&m->coords64, (size_t)m->n_nodes * sizeof(double4)) != cudaSuccess ||
            cudaMalloc(&m->coords32, (size_t)m->n_nodes * sizeof(float4)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(m->coords64);
            m->coords64 = m->coords32 = nullptr;
            return set_error(FSI_ERR_OOM, "fsi_mesh_set_coordinates: cudaMalloc failed");
        }
    }
    int64_t blocks = (m->n_nodes + 255) / 256;
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    pad_coords_kernel<<<(int)blocks, 256, 0, m->stream>>>(m->n_nodes, X, (double4 *)m->coords64,
                                                          (float4 *)m->coords32);
    return check_launch("pad coordinates kernel");
}

fsi_status fsi_mesh_set_physics(fsi_mesh *m, const fsi_physics *phys)
{
    FSI_TRY(validate_mesh(m));
    FSI_TRY(validate_physics(phys));
    m->phys = *phys;
    derive(m);
    if (m->tet) tet_set_physics(m->tet, phys);
    return FSI_OK;
}

fsi_status fsi_mesh_set_brick(fsi_mesh *m, int op, fsi_prec prec, int bx, int by, int bz,
                              int threads)
{
    FSI_TRY(validate_mesh(m));
    FSI_TRY(require_structured(m, "fsi_mesh_set_brick"));
    if (op < 0 || op > 2 || (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64))
        return set_error(FSI_ERR_ARG, "bad op or precision");
    if (bx < 1 || by < 1 || bz < 1 || threads < 32 || threads > 256 || threads % 32 != 0)
        return set_error(FSI_ERR_ARG, "bad brick %dx%dx%d / %d threads", bx, by, bz, threads);
    const size_t smem = (op == 2 ? 2 : 1) * (size_t)bx * by * bz * 8 * 4 * (prec == FSI_F32 ? 4 : 8);
    if (smem > 200 * 1024)
        return set_error(FSI_ERR_ARG, "brick %dx%dx%d needs %zu bytes of shared memory", bx, by,
                         bz, smem);
    m->brick[op][prec] = Brick{bx, by, bz, threads};
    return FSI_OK;
}

fsi_status fsi_mesh_sizes(const fsi_mesh *m, int64_t *n_nodes, int64_t *n_elems)
{
    FSI_TRY(validate_mesh(m));
    if (n_nodes) *n_nodes = m->n_nodes;
    if (n_elems) *n_elems = m->n_elems;
    return FSI_OK;
}

fsi_status fsi_stage(fsi_mesh *m, fsi_prec prec, const void *y, const void *Vn, const void *An,
                     const void *s, void *U, void *A)
{
    FSI_TRY(validate_mesh(m));
    if (!y || !Vn || !An || !U || !A)
        return set_error(FSI_ERR_ARG, "fsi_stage: NULL array argument");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(m->device);
    const int threads = 256;
    const int blocks = grid_for(m->n_nodes, threads);
    const double dt = m->phys.dt;
    if (prec == FSI_F64)
        stage_kernel<double><<<blocks, threads, 0, m->stream>>>(
            m->n_nodes, dt, m->alpha_m, m->alpha_f, m->gamma, (const vec4<double> *)y,
            (const vec4<double> *)Vn, (const vec4<double> *)An, (const double *)s,
            (vec4<double> *)U, (vec4<double> *)A);
    else
        stage_kernel<float><<<blocks, threads, 0, m->stream>>>(
            m->n_nodes, (float)dt, (float)m->alpha_m, (float)m->alpha_f, (float)m->gamma,
            (const vec4<float> *)y, (const vec4<float> *)Vn, (const vec4<float> *)An,
            (const float *)s, (vec4<float> *)U, (vec4<float> *)A);
    return check_launch("stage kernel");
}

fsi_status fsi_advance_history(fsi_mesh *m, fsi_prec prec, const void *y, void *Vn, void *An)
{
    FSI_TRY(validate_mesh(m));
    if (!y || !Vn || !An) return set_error(FSI_ERR_ARG, "fsi_advance_history: NULL argument");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(m->device);
    const int threads = 256;
    const int blocks = grid_for(m->n_nodes, threads);
    if (prec == FSI_F64)
        advance_kernel<double><<<blocks, threads, 0, m->stream>>>(
            m->n_nodes, m->phys.dt, m->gamma, (const vec4<double> *)y, (vec4<double> *)Vn,
            (vec4<double> *)An);
    else
        advance_kernel<float><<<blocks, threads, 0, m->stream>>>(
            m->n_nodes, (float)m->phys.dt, (float)m->gamma, (const vec4<float> *)y,
            (vec4<float> *)Vn, (vec4<float> *)An);
    return check_launch("advance kernel");
}

fsi_status fsi_residual(fsi_mesh *m, fsi_prec prec, const void *U, const void *A, const void *f,
                        void *R)
{
    FSI_TRY(validate_mesh(m));
    if (!U || !A || !R) return set_error(FSI_ERR_ARG, "fsi_residual: NULL array argument");
    if (R == U || R == A || (f && R == f))
        return set_error(FSI_ERR_ARG, "fsi_residual: R aliases an input");
    if (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(m->device);
    return vms_residual(m, prec, U, A, f, R);
}

fsi_status fsi_residual_jacobian_apply(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                                       const void *f, const void *x, void *R, void *Jx)
{
    FSI_TRY(validate_mesh(m));
    if (!U || !A || !x || !R || !Jx)
        return set_error(FSI_ERR_ARG, "fsi_residual_jacobian_apply: NULL array argument");
    const void *in[4] = {U, A, f, x};
    for (const void *p : in)
        if (p && (p == R || p == Jx))
            return set_error(FSI_ERR_ARG, "fsi_residual_jacobian_apply: an output aliases an input");
    if (R == Jx) return set_error(FSI_ERR_ARG, "fsi_residual_jacobian_apply: R and Jx alias");
    if (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(m->device);
    return vms_residual_jacobian(m, prec, U, A, f, x, R, Jx);
}

fsi_status fsi_jacobian_apply(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                              const void *f, const void *x, void *Jx)
{
    FSI_TRY(validate_mesh(m));
    if (!U || !A || !x || !Jx)
        return set_error(FSI_ERR_ARG, "fsi_jacobian_apply: NULL array argument");
    if (Jx == U || Jx == A || Jx == x)
        return set_error(FSI_ERR_ARG, "fsi_jacobian_apply: Jx aliases an input");
    if (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64)
        return set_error(FSI_ERR_ARG, "bad precision");
    FSI_DEVICE(m->device);
    return vms_jacobian(m, prec, U, A, f, x, Jx);
}

}  // extern "C"
