// fsi_internal.cuh -- definitions shared by the translation units of libfsi.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "fsi.h"

namespace fsi {

// ---------------------------------------------------------------- errors
fsi_status set_error(fsi_status st, const char *fmt, ...);
fsi_status check_cuda(cudaError_t e, const char *what);
fsi_status check_launch(const char *what);

#define FSI_TRY(expr)                       \
    do {                                    \
        fsi_status _st = (expr);            \
        if (_st != FSI_OK) return _st;      \
    } while (0)

#define FSI_CUDA(expr, what) FSI_TRY(::fsi::check_cuda((expr), (what)))

// ---------------------------------------------------------------- devices
// Makes `device` the calling thread's current device for the guard's
// lifetime and gives the caller's current device back when it ends, so that
// no entry point leaves the thread on another device.
class DeviceGuard {
public:
    explicit DeviceGuard(int device);
    ~DeviceGuard();
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
    fsi_status status() const { return st_; }

private:
    int prev_ = -1;
    fsi_status st_ = FSI_OK;
};

#define FSI_DEVICE(dev)                      \
    ::fsi::DeviceGuard _fsi_device_guard(dev); \
    FSI_TRY(_fsi_device_guard.status())

// Number of SMs of the current device (queried once per device).  Grid caps
// are multiples of it, so that they follow the GPU the library runs on.
int sm_count();

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device (once per kernel and device; thread-safe).
fsi_status set_smem_limit(const void *kernel, int bytes);

// ---------------------------------------------------------------- 4-vectors
// 16/32-byte aligned node records so that one node is one vector load.
template <typename T> struct alignas(4 * sizeof(T)) vec4 {
    T x, y, z, w;
};

template <typename T> __device__ __forceinline__ vec4<T> ld4(const vec4<T> *p);
template <> __device__ __forceinline__ vec4<float> ld4(const vec4<float> *p)
{
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ vec4<double> ld4(const vec4<double> *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return {a.x, a.y, b.x, b.y};
}

template <typename T> __device__ __forceinline__ void st4(vec4<T> *p, vec4<T> v) { *p = v; }

// ---------------------------------------------------------------- tuning
struct Brick {
    int bx, by, bz;  // elements per CTA along each axis
    int threads;     // CTA size (multiple of 32; 8 lanes per element)
};

struct NewtonWorkspace;
struct PressureMG;
struct TetAmg;

// ---------------------------------------------------------------- mesh
}  // namespace fsi

struct fsi_mesh {
    fsi_grid grid;
    fsi_physics phys;
    int device;
    cudaStream_t stream;
    int64_t n_nodes, n_elems;
    double alpha_m, alpha_f, gamma;
    // VMS brick schedule per [op: 0 residual, 1 jacobian, 2 both fused]
    // [compute type: FSI_F64, FSI_F32, FSI_DF64]
    fsi::Brick brick[3][3];
    // scratch: per-brick node-block partial sums of the VMS operators
    void *vms_scratch;
    size_t vms_scratch_bytes;
    // scratch: cell fill counters [E+1] + scan scratch + misc counters;
    // hash_clean: the counters are known to be all zero
    int32_t *hash_fill;
    int32_t *scan_tmp;
    int64_t scan_tmp_len;
    bool hash_clean;
    // grow-only point scratch of the cell table ((point, cell) pairs)
    int2 *pt_tmp;
    int64_t pt_tmp_cap;
    int64_t *dev_counters;  // [0] outside count, [1] error flag
    // scratch: per-cell corner sums of the spreading operator [E][8][3]
    void *spread_scratch;
    size_t spread_scratch_bytes;
    // Newton / Krylov workspace (newton.cu), created on first use
    fsi::NewtonWorkspace *newton;
    // pressure multigrid hierarchy of the Schur preconditioner (pmg.cu)
    fsi::PressureMG *pmg;
    // mapped grid: node coordinates padded to [n][4], FP64 and FP32 copies
    // (null on the uniform grid)
    void *coords64, *coords32;
    // mapped grid: per-Gauss-point geometry tables [double, float, double-float],
    // built on first use, dropped when the coordinates change (vms.cu)
    void *map_geo[3];
    // unstructured tetrahedral mesh behind this handle (fsi_mesh_create_tet);
    // null for the structured grid
    fsi_tetmesh *tet;
    // algebraic multigrid of the pressure Schur approximation on the
    // tetrahedral mesh, or on the structured grid when pressure_amg is set
    // (amg.cu); built on first use, dropped when the coordinates change
    fsi::TetAmg *amg;
    bool pressure_amg;
};

namespace fsi {

// the pressure block of the Schur preconditioner is the algebraic multigrid
inline bool uses_amg(const fsi_mesh *m) { return m->tet != nullptr || m->pressure_amg; }

fsi_status validate_mesh(const fsi_mesh *m);
fsi_status ensure_vms_scratch(fsi_mesh *m, const Brick &b, size_t elem_bytes);
size_t vms_scratch_bytes_for(const fsi_mesh *m, const Brick &b, size_t elem_bytes);
fsi_status ensure_spread_scratch(fsi_mesh *m, size_t bytes);
void destroy_newton_workspace(fsi_mesh *m);

// pressure multigrid (pmg.cu)
fsi_status pmg_ensure(fsi_mesh *m);
fsi_status pmg_set_faces(fsi_mesh *m, const int faces[6]);
template <typename T> fsi_status pmg_vcycle(fsi_mesh *m, const T *b, T *x);
// the V-cycle as the pressure block of the Schur preconditioner: the result
// x goes straight into the pressure slot of z [n][4] as x / sigma, or
// v [n][4]'s pressure where mask [n][4] (uint8, may be null) fixes it; false
// (nothing launched) when the hierarchy has a single level
template <typename T>
fsi_status pmg_vcycle_schur(fsi_mesh *m, const T *b, T *z, const T *v, const uint8_t *mask,
                            T inv_sigma, bool *done);
void *pmg_fine_buffer(fsi_mesh *m, int which);
void destroy_pmg(fsi_mesh *m);

// pressure algebraic multigrid on a tetrahedral mesh (amg.cu); the
// elimination set is one flag per node, or derived from a step's Dirichlet
// mask (boundary nodes with free velocity, nodes with fixed pressure)
fsi_status amg_set_eliminated(fsi_mesh *m, const std::vector<uint8_t> &elim);
fsi_status amg_set_from_mask(fsi_mesh *m, const uint8_t *mask);
template <typename T> fsi_status amg_vcycle(fsi_mesh *m, const T *b, T *x);
void *amg_fine_buffer(fsi_mesh *m, int which);
fsi_status amg_level_sizes(fsi_mesh *m, int32_t *n_levels, int64_t *n);
fsi_status amg_apply(fsi_mesh *m, fsi_prec prec, int level, const void *x, void *y);
fsi_status amg_restrict(fsi_mesh *m, fsi_prec prec, int level, const void *r, void *b);
fsi_status amg_prolong_add(fsi_mesh *m, fsi_prec prec, int level, const void *xc, void *x);
fsi_status amg_smooth(fsi_mesh *m, fsi_prec prec, int level, int degree, const void *b, void *x,
                      int from_zero);
void destroy_amg(fsi_mesh *m);

// immersed hyperelastic solid (solid.cu)
fsi_status solid_residual_impl(fsi_solid *b, const double *u_af, const double *v_af,
                               const double *a_am, const double *u_n, const double g[3], double *R);
template <typename T>
fsi_status solid_tangent_impl(fsi_solid *b, const T *u_af, const double *u_n, const T *x, T *Jx);
fsi_status solid_stage_impl(fsi_solid *b, const double *u, const double *v, const double *a,
                            const double *a1, double *u_af, double *v_af, double *a_am);
int64_t solid_nodes(const fsi_solid *b);

// tensor-core GEMM of the network's training (mlp_gemm.cu):
// C[M x N] = epi(op(A) op(B)), FP32 operands rounded to BF16, FP32 accumulation;
// op(A) = A [M][K] (lda) or, with transA, A^T of A [K][M]; op(B) = B [K][N]
// (ldb) or, with transB, B^T of B [N][K].  N <= 256.  work: the split-K
// workspace (tc_gemm_work_floats() floats); err: a device flag raised when a
// tensor-core wait runs out.
enum TcEpi { TC_EPI_STORE = 0, TC_EPI_BIAS = 1, TC_EPI_BIAS_RELU = 2, TC_EPI_MASK = 3 };
struct TcGemm {
    int M, N, K;
    const float *A;
    int64_t lda;
    int transA;
    const float *B;
    int64_t ldb;
    int transB;
    float *C;
    int64_t ldc;
    int epi;
    const float *bias;  // [N] for TC_EPI_BIAS / TC_EPI_BIAS_RELU
    float *Cpre;        // pre-activation output for TC_EPI_BIAS_RELU (may be null)
    const float *mask;  // [M x N] (ldc) for TC_EPI_MASK: C *= (mask > 0)
    int BN;             // set by tc_gemm: N rounded up to a multiple of 16
};
size_t tc_gemm_work_floats();
fsi_status tc_gemm(cudaStream_t s, const TcGemm &g, float *work, int *err);

// fused tensor-core inference of the initial-guess network (mlp_tc.cu)
size_t mlp_tc_packed_bytes();
fsi_status mlp_predict_tc(cudaStream_t s, int device, const fsi_grid &g, int64_t n,
                          const float *params, const float *in_mean, const float *in_std,
                          const float *out_mean, const float *out_std, const double *Vn,
                          const double *y, const double *d1, const double *d2, double *y0,
                          void *packed, int *dev_err);

// the coupled Jacobian (newton.cu) at st->y applied to k FP32 vectors after
// one linearisation; used by the learned guess's fitted predictor
// Nodal diagonal blocks of the VMS Jacobian at (U, A, f) on the uniform
// grid (diag.cu): blocks [n][4][4] row-major in the compute type (FSI_F64 or
// FSI_F32 arrays), rows and columns 0..ncols-1 (3: velocity, 4: with
// pressure) overwritten, the rest zero.  Mesh's stream.
fsi_status vms_diag_blocks(fsi_mesh *m, fsi_prec prec, int ncols, const void *U, const void *A,
                           const void *f, void *blocks);

// F[a].xyz = dsq sum_B w_B N_a(xi_B)^2 (the diagonal of C W C^T scaled by
// dsq; dlm.cu), over the points of the cell table, deterministic.
template <typename T>
fsi_status spread_mass_diag(fsi_mesh *mesh, int64_t m, const T *xi, const int32_t *cell_start,
                            const int32_t *perm, const T *w, double dsq, T *F);

// the checks fsi_newton_step makes of a step state (newton.cu)
fsi_status validate_step_state(const fsi_mesh *mesh, const fsi_step_state *st);

fsi_status coupled_jacobian_f32(fsi_mesh *mesh, const fsi_step_state *st, int k,
                                const float *const *x, float *const *Jx, double *R_fit = nullptr);

// VMS operators (vms.cu)
fsi_status vms_residual(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                        const void *f, void *R);
fsi_status vms_jacobian(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                        const void *f, const void *x, void *Jx);
fsi_status vms_residual_jacobian(fsi_mesh *m, fsi_prec prec, const void *U, const void *A,
                                 const void *f, const void *x, void *R, void *Jx);

// tetrahedral meshes (tet.cu): stream and physics follow the owning fsi_mesh;
// a distance-2 node colouring (no two nodes of one element share a colour)
// for probing the nodal diagonal blocks
void tet_set_stream(fsi_tetmesh *t, cudaStream_t s);
void tet_set_physics(fsi_tetmesh *t, const fsi_physics *p);
const int32_t *tet_colors(const fsi_tetmesh *t, int *n_colors);
// host copies of the node coordinates [n][3] and elements [E][4], and the
// bounding box (synchronises the mesh stream)
fsi_status tet_download(fsi_tetmesh *t, std::vector<double> &X, std::vector<int32_t> &tets,
                        double box_lo[3], double box_hi[3]);
fsi_status require_structured(const fsi_mesh *m, const char *what);

// cell -> points table (dlm.cu): from per-cell counts in fill[0..E), an
// exclusive scan into cell_start[E+1], a scatter of the points into perm and
// a per-cell sort by point index (outside points last).  fill is counted
// back down as the slots are handed out and is all zero again on return;
// scan_tmp holds cell_table_scan_ints(E) ints, all zero before the first
// call, which every call leaves so.
int64_t cell_table_scan_ints(int64_t E);
// With tmp (m (point, cell) pairs of scratch), the locate kernel has left
// each point's arrival slot in perm and counted outside points in fill[E];
// the slices are then ordered by a rank pass from tmp into perm.  Without
// tmp, fill[E] is unused and the slices are sorted in place in perm.
fsi_status build_cell_table(cudaStream_t s, int64_t E, int64_t m, const int32_t *elem,
                            int32_t *fill, int32_t *scan_tmp, int32_t *cell_start, int32_t *perm,
                            int2 *tmp = nullptr);

}  // namespace fsi
