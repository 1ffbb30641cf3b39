// vms.cu -- matrix-free VMS residual and Jacobian-vector product on the
// uniform Q1-Q1 hex grid (Sec. 2.1 / 2.4 of the paper; form of Bazilevs et
// al. 2007).
//
// Layout of the work:
//   * One CTA per brick of bx*by*bz elements.  Eight consecutive lanes own one
//     element; lane g (bits gx, gy, gz) is first "node a = g" (it loads that
//     node's record) and then "Gauss point g".  On the uniform grid the Q1
//     basis is a tensor product of 1D linear functions, so the values and
//     gradients at the 2x2x2 Gauss points follow from the nodal values by
//     three butterfly stages over the lane bits (shfl.xor 1, 2, 4), and the
//     test-function projection is the transposed butterfly.  No shape-function
//     tables, no smem bank traffic for evaluation.
//   * After the projection lane g holds the element's contribution to its
//     local node g.  Contributions go to shared memory per element; after the
//     brick is done every node of the brick's node block sums its (<= 8)
//     element contributions in a fixed corner order (no atomics).
//   * Bricks share the nodes on their faces, so each brick writes its whole
//     node block to scratch, and a second kernel sums, for every node, the
//     blocks that contain it in a fixed brick order.  The result is
//     deterministic (bitwise reproducible) and atomic-free.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "fsi_internal.cuh"

#include "vms_device.cuh"

namespace fsi {
namespace {

using namespace vmsd;

template <typename T, bool JAC, bool MAPPED, bool FUSED = false>
__global__ void __launch_bounds__(256) vms_brick_kernel(const VmsArgs<T> P)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    brick_body<T, JAC, MAPPED, FUSED>(P, blockIdx.x, reinterpret_cast<vec4<T> *>(smem_raw));
}

// The same, held to 128 registers (two 256-thread CTAs per SM): used for the
// mapped double-float kernels, whose Jacobian otherwise takes more registers
// and runs 1.2x slower at one CTA per SM.
template <typename T, bool JAC, bool MAPPED, bool FUSED = false>
__global__ void __launch_bounds__(256, 2) vms_brick_kernel_capped(const VmsArgs<T> P)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    brick_body<T, JAC, MAPPED, FUSED>(P, blockIdx.x, reinterpret_cast<vec4<T> *>(smem_raw));
}

// Geometry table of a mapped grid: 8 lanes per element (lane = node, then
// Gauss point), the same butterfly as the VMS kernels.  The loop bound is
// uniform over the block, so every lane reaches every shuffle.
template <typename T>
__global__ void __launch_bounds__(256) mapped_geo_kernel(const VmsArgs<T> P,
                                                         typename GeoStore<T>::type *tab)
{
    const int g = threadIdx.x & 7;
    const int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
    const T sx = gx ? T(0.5f) : T(-0.5f), sy = gy ? T(0.5f) : T(-0.5f),
            sz = gz ? T(0.5f) : T(-0.5f);
    const int64_t E = (int64_t)P.Nx * P.Ny * P.Nz;
    const int64_t NX1 = P.Nx + 1, NXY1 = NX1 * (P.Ny + 1);
    const int64_t per_block = blockDim.x >> 3, stride = (int64_t)gridDim.x * per_block;
    for (int64_t base = blockIdx.x * per_block; base < E; base += stride) {
        const int64_t e = base + (threadIdx.x >> 3);
        const bool valid = e < E;
        const int64_t ex = valid ? e % P.Nx : 0, ey = valid ? (e / P.Nx) % P.Ny : 0,
                      ez = valid ? e / ((int64_t)P.Nx * P.Ny) : 0;
        const int64_t node = (ex + gx) + NX1 * (ey + gy) + NXY1 * (ez + gz);
        const vec4<T> xc = valid ? load_c<T>(P.Xc + node)
                                 : vec4<T>{gx ? T(1) : T(0), gy ? T(1) : T(0), gz ? T(1) : T(0), T(0)};
        T out[kMapGeo];
        mapped_geometry<false>(xc, sx, sy, sz, out);
        if (valid)
#pragma unroll
            for (int k = 0; k < kMapGeo; ++k) tab[e * (kMapGeo * 8) + 8 * k + g] = geo_st(out[k]);
    }
}

// index of the compute type in fsi_mesh::brick (its fsi_prec)
template <typename T> constexpr int prec_slot()
{
    return std::is_same<T, double>::value ? FSI_F64
                                          : (std::is_same<T, float>::value ? FSI_F32 : FSI_DF64);
}

template <typename T> constexpr int geo_slot()
{
    return std::is_same<T, double>::value ? 0 : (std::is_same<T, float>::value ? 1 : 2);
}

// the geometry table of compute type T for the current coordinates, built on
// first use (it allocates: not inside a stream capture)
template <typename T> fsi_status ensure_map_geo(fsi_mesh *m, const VmsArgs<T> &P)
{
    void *&tab = m->map_geo[geo_slot<T>()];
    if (tab) return FSI_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FSI_CUDA(cudaStreamIsCapturing(m->stream, &cap), "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return set_error(FSI_ERR_ARG, "mapped-grid geometry table: first use of this compute "
                                      "type inside a stream capture");
    const size_t bytes = (size_t)m->n_elems * kMapGeo * 8 * sizeof(typename GeoStore<T>::type);
    if (cudaMalloc(&tab, bytes) != cudaSuccess) {
        cudaGetLastError();
        tab = nullptr;
        return set_error(FSI_ERR_OOM, "mapped-grid geometry table: cudaMalloc of %zu bytes failed",
                         bytes);
    }
    int64_t blocks = (m->n_elems + 31) / 32;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    mapped_geo_kernel<T><<<(int)blocks, 256, 0, m->stream>>>(P, (typename GeoStore<T>::type *)tab);
    return check_launch("mapped geometry kernel");
}

template <typename T, bool FUSED = false> __global__ void vms_gather_kernel(const VmsArgs<T> P)
{
    const int n = (P.Nx + 1) * (P.Ny + 1) * (P.Nz + 1);
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n;
         node += gridDim.x * blockDim.x)
        gather_node<T, FUSED>(P, node);
}

// FUSED: the residual (R) and the Jacobian apply (out) at the same state in
// one pass; the brick schedule is op 2's, the shared memory and the node-block
// scratch hold both operators' contributions
template <typename T, bool JAC, bool MAPPED, bool FUSED = false>
fsi_status launch_geo(fsi_mesh *m, const void *U, const void *A, const void *f, const void *x,
                      void *out, void *R = nullptr)
{
    using S = typename StorageOf<T>::type;
    const Brick &b = m->brick[FUSED ? 2 : (JAC ? 1 : 0)][prec_slot<T>()];
    FSI_TRY(ensure_vms_scratch(m, b, (FUSED ? 2 : 1) * sizeof(T)));
    VmsArgs<T> P = make_args<T>(m, b, U, A, f, x, out);
    if constexpr (MAPPED) {
        FSI_TRY(ensure_map_geo<T>(m, P));
        P.geo = (const typename GeoStore<T>::type *)m->map_geo[geo_slot<T>()];
    }
    const int nbricks = P.nbx * P.nby * P.nbz;
    if constexpr (FUSED) {
        P.blocks2 = P.blocks + (size_t)nbricks * (b.bx + 1) * (b.by + 1) * (b.bz + 1);
        P.out2 = (vec4<S> *)R;
    }
    const size_t smem = (FUSED ? 2 : 1) * (size_t)vmsd::rel_records(b.bx * b.by * b.bz) * sizeof(vec4<S>);
    void (*kernel)(const VmsArgs<T>);
    if constexpr (MAPPED && std::is_same<T, df64>::value)
        kernel = vms_brick_kernel_capped<T, JAC, MAPPED, FUSED>;
    else
        kernel = vms_brick_kernel<T, JAC, MAPPED, FUSED>;
    FSI_TRY(set_smem_limit((const void *)kernel, 200 * 1024));
    kernel<<<nbricks, b.threads, smem, m->stream>>>(P);
    FSI_TRY(check_launch("vms brick kernel"));
    const int threads = 256;
    int64_t nb = (m->n_nodes + threads - 1) / threads;
    if (nb > sm_count() * 32) nb = sm_count() * 32;
    vms_gather_kernel<T, FUSED><<<(int)nb, threads, 0, m->stream>>>(P);
    return check_launch("vms gather kernel");
}

// the mapped-grid kernels take the geometry of every Gauss point from a table
// built from the node coordinates (set by fsi_mesh_set_coordinates)
template <typename T, bool JAC>
fsi_status launch(fsi_mesh *m, const void *U, const void *A, const void *f, const void *x,
                  void *out)
{
    if (m->coords64) return launch_geo<T, JAC, true>(m, U, A, f, x, out);
    return launch_geo<T, JAC, false>(m, U, A, f, x, out);
}

template <typename T>
fsi_status launch_fused(fsi_mesh *m, const void *U, const void *A, const void *f, const void *x,
                        void *R, void *Jx)
{
    if (m->coords64) return launch_geo<T, true, true, true>(m, U, A, f, x, Jx, R);
    return launch_geo<T, true, false, true>(m, U, A, f, x, Jx, R);
}

// candidate brick shapes of the single-mesh autotuner: the default, smaller
// bricks (more bricks per wave of resident CTAs on small grids), flatter and
// longer ones, and 128-thread CTAs (more CTAs per SM)
const Brick kMeshBricks[] = {
    {8, 8, 4, 256}, {8, 4, 4, 256}, {8, 8, 2, 256}, {4, 4, 4, 256}, {4, 4, 8, 256},
    {16, 4, 4, 256}, {8, 4, 4, 128}, {4, 4, 4, 128}, {8, 4, 2, 128}, {4, 4, 2, 128},
};

template <typename S> __global__ void fill_state_kernel(int64_t n, vec4<S> *U, vec4<S> *A, vec4<S> *x)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        U[i] = {S(0.5), S(-0.25), S(0.125), S(1)};
        A[i] = {S(0), S(0), S(0), S(1)};  // s = 1
        x[i] = {S(1), S(1), S(1), S(1)};
    }
}

// seconds per launch of one operator with the mesh's current brick: one
// warm-up launch, then reps launches between CUDA events
template <typename T>
fsi_status time_op(fsi_mesh *m, int op, int reps, const void *U, const void *A, const void *x,
                   void *out, void *R, cudaEvent_t e0, cudaEvent_t e1, double *seconds)
{
    auto run = [&]() {
        if (op == 2) return launch_fused<T>(m, U, A, nullptr, x, R, out);
        return op ? launch<T, true>(m, U, A, nullptr, x, out)
                  : launch<T, false>(m, U, A, nullptr, nullptr, out);
    };
    FSI_TRY(run());
    FSI_CUDA(cudaEventRecord(e0, m->stream), "event");
    for (int r = 0; r < reps; ++r) FSI_TRY(run());
    FSI_CUDA(cudaEventRecord(e1, m->stream), "event");
    FSI_CUDA(cudaEventSynchronize(e1), "event sync");
    float ms = 0.0f;
    FSI_CUDA(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    *seconds = 1e-3 * ms / reps;
    return FSI_OK;
}

template <typename T> fsi_status autotune(fsi_mesh *m, int op, int reps, fsi_tune_report *rep)
{
    using S = typename StorageOf<T>::type;
    const int slot = prec_slot<T>();
    const Brick start = m->brick[op][slot];
    const size_t bytes = (size_t)m->n_nodes * sizeof(vec4<S>);
    void *buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fsi_status st = FSI_OK;
    for (void *&b : buf)
        if (cudaMalloc(&b, bytes) != cudaSuccess) {
            cudaGetLastError();
            st = set_error(FSI_ERR_OOM, "fsi_mesh_autotune: cudaMalloc failed");
        }
    if (st == FSI_OK &&
        (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = set_error(FSI_ERR_CUDA, "fsi_mesh_autotune: cudaEventCreate failed");
    double best = 1e30;
    Brick best_brick = start;
    int tried = 0;
    if (st == FSI_OK) {
        fill_state_kernel<S><<<sm_count() * 4, 256, 0, m->stream>>>(m->n_nodes, (vec4<S> *)buf[0],
                                                             (vec4<S> *)buf[1], (vec4<S> *)buf[2]);
        st = check_launch("autotune fill");
    }
    for (const Brick &cand : kMeshBricks) {
        if (st != FSI_OK) break;
        m->brick[op][slot] = cand;
        double t = 0.0;
        st = time_op<T>(m, op, reps, buf[0], buf[1], buf[2], buf[3], buf[4], e0, e1, &t);
        if (st != FSI_OK) break;
        if (tried < FSI_TUNE_MAX_CANDIDATES) {
            rep->cand_bx[tried] = cand.bx;
            rep->cand_by[tried] = cand.by;
            rep->cand_bz[tried] = cand.bz;
            rep->cand_ctas[tried] = cand.threads;
            rep->cand_seconds[tried] = t;
        }
        ++tried;
        if (t < best) {
            best = t;
            best_brick = cand;
        }
    }
    m->brick[op][slot] = st == FSI_OK ? best_brick : start;
    cudaStreamSynchronize(m->stream);
    for (void *b : buf) cudaFree(b);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != FSI_OK) return st;
    rep->n_candidates = tried < FSI_TUNE_MAX_CANDIDATES ? tried : FSI_TUNE_MAX_CANDIDATES;
    rep->bx = best_brick.bx;
    rep->by = best_brick.by;
    rep->bz = best_brick.bz;
    rep->threads = best_brick.threads;
    rep->ctas_per_sm = 0;
    rep->seconds = best;
    return FSI_OK;
}

}  // namespace

fsi_status vms_residual(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                        const void *f, void *R)
{
    if (m->tet) return fsi_tet_residual(m->tet, prec, U, A, f, R);
    if (prec == FSI_F64) return launch<double, false>(m, U, A, f, nullptr, R);
    if (prec == FSI_DF64) return launch<df64, false>(m, U, A, f, nullptr, R);
    return launch<float, false>(m, U, A, f, nullptr, R);
}

fsi_status vms_residual_jacobian(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                                 const void *f, const void *x, void *R, void *Jx)
{
    if (m->tet) {
        FSI_TRY(fsi_tet_residual(m->tet, prec, U, A, f, R));
        return fsi_tet_jacobian_apply(m->tet, prec, U, A, f, x, Jx);
    }
    if (prec == FSI_F64) return launch_fused<double>(m, U, A, f, x, R, Jx);
    if (prec == FSI_DF64) return launch_fused<df64>(m, U, A, f, x, R, Jx);
    return launch_fused<float>(m, U, A, f, x, R, Jx);
}

fsi_status vms_jacobian(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                        const void *f, const void *x, void *Jx)
{
    if (m->tet) return fsi_tet_jacobian_apply(m->tet, prec, U, A, f, x, Jx);
    if (prec == FSI_F64) return launch<double, true>(m, U, A, f, x, Jx);
    if (prec == FSI_DF64) return launch<df64, true>(m, U, A, f, x, Jx);
    return launch<float, true>(m, U, A, f, x, Jx);
}

}  // namespace fsi

using namespace fsi;

extern "C" fsi_status fsi_mesh_autotune(fsi_mesh *mesh, int op, fsi_prec prec, int reps,
                                        fsi_tune_report *report)
{
    FSI_TRY(validate_mesh(mesh));
    FSI_TRY(require_structured(mesh, "fsi_mesh_autotune"));
    if (op < 0 || op > 2 || reps < 1 || !report ||
        (prec != FSI_F64 && prec != FSI_F32 && prec != FSI_DF64))
        return set_error(FSI_ERR_ARG, "fsi_mesh_autotune: bad arguments");
    FSI_DEVICE(mesh->device);
    std::memset(report, 0, sizeof *report);
    if (prec == FSI_F64) return autotune<double>(mesh, op, reps, report);
    if (prec == FSI_DF64) return autotune<df64>(mesh, op, reps, report);
    return autotune<float>(mesh, op, reps, report);
}

