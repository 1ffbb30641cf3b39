/*
 * fsi.h -- C ABI of the GB300 immersed-FSI hot-path library (libfsi.so).
 *
 * The library evaluates, on one GPU, the data-parallel operators of the
 * monolithic fictitious-domain / distributed-Lagrange-multiplier FSI method
 * of arxiv 2601.08266 (Black et al., "An open-source computational framework
 * for immersed fluid-structure interaction modeling using FEBio and MFEM"):
 *
 *   - the VMS-stabilised incompressible Navier-Stokes residual on a uniform
 *     Q1-Q1 hexahedral background grid and its consistent Jacobian-vector
 *     product (Sec. 2.1, Eq. fluid_weak_form, and the reduced block system of
 *     Sec. 2.4);
 *   - the coupling operators of Sec. 2.3: locating solid points in fluid
 *     elements, interpolation u = C^T V (Eq. nodal_solid_velo) and spreading
 *     F = C lambda (Eq. fsi_constraint_matrix);
 *   - the Newton step on the reduced system (Sec. 2.4).
 *
 * Conventions (apply to every entry point unless its comment says otherwise):
 *   - Every array argument is a DEVICE pointer on the mesh's device, owned by
 *     the caller, contiguous, row-major.  Nodal fields are [n][4] with
 *     n = (Nx+1)(Ny+1)(Nz+1) nodes numbered lexicographically, x fastest:
 *     node(i,j,k) = i + (Nx+1)*(j + (Ny+1)*k).  Slots are (vx, vy, vz, p) for
 *     velocity-pressure fields and (ax, ay, az, s) for the acceleration field
 *     A, whose 4th slot carries the interface scaling s of Sec. 2.1 when the
 *     mesh was created with has_s != 0 (it is ignored otherwise).
 *     Elements are numbered e = ex + Nx*(ey + Ny*ez).
 *   - fsi_prec selects the element type of the floating-point arrays of that
 *     call: FSI_F64 = double, FSI_F32 = float.  FSI_DF64 takes double arrays
 *     and computes in double-float arithmetic (pairs of floats on the FP32
 *     units, about 2^-44 relative per operation); the calls that accept it
 *     say so.  Point coordinates X are always double.
 *   - Calls are asynchronous and stream-ordered on the mesh's stream, except
 *     where a comment says the call synchronises.  Arrays must stay valid
 *     until the stream has passed the call.
 *   - Invalid arguments return FSI_ERR_ARG without launching anything; every
 *     error also sets a thread-local message returned by fsi_last_error().
 *     No C++ exception crosses this interface.
 *   - The library allocates device memory only inside fsi_mesh objects (its
 *     scratch); it never frees caller memory.
 */
#ifndef FSI_H
#define FSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FSI_OK = 0,
    FSI_ERR_ARG = 1,      /* invalid argument; nothing was launched          */
    FSI_ERR_CUDA = 2,     /* a CUDA runtime call or kernel launch failed      */
    FSI_ERR_OOM = 3,      /* device allocation failed                         */
    FSI_ERR_OUTSIDE = 4,  /* strict locate: some point lies outside the grid  */
    FSI_ERR_NOCONV = 5,   /* Newton did not reach its tolerance               */
    FSI_ERR_TIMEOUT = 6,  /* a bounded device wait gave up                    */
    FSI_ERR_NAN = 7       /* a non-finite norm was met                        */
} fsi_status;

/* FSI_F64: IEEE double arrays and arithmetic.  FSI_F32: IEEE float.
 * FSI_DF64: IEEE double arrays, arithmetic in double-float (pairs of floats,
 * about 48 significant bits) on the FP32 pipe -- GB300 runs FP32 ~70x faster
 * than FP64; accepted by fsi_residual and fsi_jacobian_apply, whose results
 * then agree with FP64 to ~1e-13 relative.                                 */
typedef enum { FSI_F64 = 0, FSI_F32 = 1, FSI_DF64 = 2 } fsi_prec;

/* Opaque handle: grid, physics, stream, tuning and library-owned scratch. */
typedef struct fsi_mesh fsi_mesh;

/* Uniform axis-aligned hexahedral grid: N[k] elements of size h[k] along
 * axis k starting at x0[k] (the unfitted background fluid mesh, Sec. 2). */
typedef struct {
    int32_t N[3];
    double x0[3];
    double h[3];
} fsi_grid;

/* Fluid and time-integration parameters.
 *   rho, mu  fluid density and dynamic viscosity (Eq. fluid_weak_form);
 *   dt       time step; rho_inf spectral radius of the generalized-alpha
 *            method (Sec. 2.4) giving alpha_m = (3-rho_inf)/(2(1+rho_inf)),
 *            alpha_f = 1/(1+rho_inf), gamma = 1/2 + alpha_m - alpha_f;
 *   C_I, C_T constants of tau_m (Sec. 2.1; the paper uses 36 and 4);
 *   has_s    nonzero: the 4th slot of A holds the nodal scaling field s of
 *            Sec. 2.1, interpolated like the pressure; zero: s = 1.        */
typedef struct {
    double rho, mu, dt, rho_inf, C_I, C_T;
    int32_t has_s;
    int32_t reserved;
} fsi_physics;

/* Create a mesh handle on CUDA device `device`, issuing work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * Allocates the handle's scratch.  Returns FSI_ERR_ARG for N[k] < 1,
 * h[k] <= 0, rho <= 0, mu < 0, dt <= 0, or a grid with more than 2^31-1
 * nodes; FSI_ERR_OOM when scratch cannot be allocated.                    */
fsi_status fsi_mesh_create(const fsi_grid *grid, const fsi_physics *phys, int device,
                           void *cuda_stream, fsi_mesh **out);

/* Release the handle and its scratch (synchronises its stream).  NULL ok. */
void fsi_mesh_destroy(fsi_mesh *mesh);

/* Change the stream subsequent calls are issued on. */
fsi_status fsi_mesh_set_stream(fsi_mesh *mesh, void *cuda_stream);

/* Replace the physics parameters (same validation as fsi_mesh_create). */
fsi_status fsi_mesh_set_physics(fsi_mesh *mesh, const fsi_physics *phys);

/* Number of nodes n and elements E of the mesh (host outputs, may be NULL). */
fsi_status fsi_mesh_sizes(const fsi_mesh *mesh, int64_t *n_nodes, int64_t *n_elems);

/* Thread-local description of the last error on this thread ("" if none). */
const char *fsi_last_error(void);

/* Generalized-alpha stage values (Sec. 2.4).  From the unknown
 * y = (Vdot_{n+1}, P_{n+1}) [n][4] and the history Vn = (V_n, -) and
 * An = (Vdot_n, -) [n][4]:
 *   V_{n+1}     = V_n + dt Vdot_n + gamma dt (Vdot_{n+1} - Vdot_n)
 *   U = (V_n + alpha_f (V_{n+1} - V_n),  P_{n+1})
 *   A = (Vdot_n + alpha_m (Vdot_{n+1} - Vdot_n),  s)
 * s [n] (same precision) fills A's 4th slot; NULL writes 1.  Slot 4 of Vn
 * and An is ignored.                                                       */
fsi_status fsi_stage(fsi_mesh *mesh, fsi_prec prec, const void *y, const void *Vn,
                     const void *An, const void *s, void *U, void *A);

/* End of a time step (generalized alpha, Sec. 2.4): from the converged
 * y = (Vdot_{n+1}, P_{n+1}) update the history in place,
 *   Vn <- V_{n+1} = V_n + dt Vdot_n + gamma dt (Vdot_{n+1} - Vdot_n),
 *   An <- Vdot_{n+1}  (velocity slots; slot 4 untouched).                  */
fsi_status fsi_advance_history(fsi_mesh *mesh, fsi_prec prec, const void *y, void *Vn, void *An);

/* VMS residual R [n][4] (Sec. 2.1): the Galerkin form of Eq. fluid_weak_form
 * with the residual-based VMS terms (SUPG, PSPG, LSIC, cross and Reynolds
 * stress) of Bazilevs et al. 2007, tau_m and tau_c of Sec. 2.1, 2x2x2 Gauss
 * quadrature.  U = (v, p) and A = (a, s) are the stage values; f [n][4]
 * (slots 0..2) is a nodal body force or NULL.  Rows 0..2 of each node are
 * the momentum residual R^{f,m}, row 3 the continuity residual R^{f,c}.
 * Boundary conditions are not applied (natural traction-free boundaries).
 * R is overwritten; it must not alias any input.  Deterministic: the same
 * inputs give bitwise the same R.                                          */
fsi_status fsi_residual(fsi_mesh *mesh, fsi_prec prec, const void *U, const void *A,
                        const void *f, void *R);

/* Consistent Jacobian-vector product Jx [n][4] of fsi_residual with respect
 * to the unknown y = (Vdot_{n+1}, P_{n+1}) of the reduced system of Sec. 2.4
 * at the stage (U, A): the exact directional derivative of R in the
 * direction dU = (alpha_f gamma dt x_v, x_p), dA = (alpha_m x_v, 0),
 * including the dependence of tau_m and tau_c on v.  f as in fsi_residual
 * (the Jacobian depends on it through the strong residual inside the fine
 * scales u').  Jx must not alias any input.  Deterministic.               */
fsi_status fsi_jacobian_apply(fsi_mesh *mesh, fsi_prec prec, const void *U, const void *A,
                              const void *f, const void *x, void *Jx);

/* Both operators at one stage in one pass: R as fsi_residual and Jx as
 * fsi_jacobian_apply, from one evaluation of U and A and one base state
 * (tau_m, tau_c, fine scales) per Gauss point.  In FSI_DF64 the results are
 * bitwise those of the two separate calls under the same brick schedule (the
 * element-to-node sums follow the bricks); in FSI_F64 and FSI_F32 they agree
 * with them to rounding (the compiler may contract differently).  The brick
 * schedule is op 2 of fsi_mesh_set_brick / fsi_mesh_autotune (default 8x4x4
 * elements, 256 threads: the pass needs twice the shared memory per brick).  On a
 * tetrahedral mesh the two operators run one after the other.  Neither
 * output may alias an input or the other output.                          */
fsi_status fsi_residual_jacobian_apply(fsi_mesh *mesh, fsi_prec prec, const void *U,
                                       const void *A, const void *f, const void *x, void *R,
                                       void *Jx);

/* Point location on the grid plus the cell -> points table (the point search
 * that builds C^lambda, Sec. 3 and Algorithm 1).  For each of the m points
 * X [m][3] (double):  t_k = (X_k - x0_k)/h_k; the point is outside unless
 * 0 <= t_k <= N_k for every k (NaN counts as outside); otherwise
 * e_k = min(floor(t_k), N_k - 1), elem = e_x + Nx (e_y + Ny e_z) and
 * xi_k = 2 (t_k - e_k) - 1 in [-1, 1].  Outside points get elem = -1 and
 * xi = 0.  cell_start [E+1] and perm [m] (int32, may both be NULL to skip)
 * receive a stable counting sort of the inside points by element:
 * the points of element e are perm[cell_start[e] .. cell_start[e+1]) in
 * increasing index order, followed in perm by the outside points in
 * increasing index order.  n_outside (HOST pointer, may be NULL) receives
 * the number of outside points; passing it makes the call synchronise.
 * strict != 0 returns FSI_ERR_OUTSIDE (after completing all outputs) when
 * some point is outside.  m may be 0.  m must be < 2^31.
 * On a structured mesh the table uses a point scratch of the mesh (8 bytes
 * per point) that grows on the first call with a table and on any later call
 * with more points than before: that call allocates (cudaMalloc, FSI_ERR_OOM
 * if it fails) and so must not be the first such call inside a stream
 * capture.  Calls with at most as many points as an earlier one allocate
 * nothing.  Between calls perm's contents are the caller's; during the call
 * perm also serves as scratch before receiving the table.                  */
fsi_status fsi_locate(fsi_mesh *mesh, int64_t m, const double *X, int32_t *elem, double *xi,
                      int32_t *cell_start, int32_t *perm, int64_t *n_outside, int strict);

/* fsi_locate without any device allocation (the paper has no counterpart).
 * Same inputs, outputs, ordering and errors as fsi_locate, bit for bit, but
 * it needs no fsi_mesh: the grid is passed by value and the work is issued
 * on `cuda_stream` of CUDA device `device`.  It exists for callers that must
 * not call cudaMalloc: code that runs inside a host application whose memory
 * manager owns all device memory, and loops that cannot pay the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree.
 * Its scratch (per-cell counters, scan tile sums, outside counter) lives in
 * one static device array of about 16 MB that every device which loads the
 * library holds until the process exits; grids with more than 4,000,000
 * cells are rejected with FSI_ERR_ARG before anything is launched.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture
 * begins.  The address is kept per device for the life of the process: it
 * is not valid across a reset of the device's primary context
 * (cudaDeviceReset), after which this entry point must not be called.
 * Grids are checked against the limit factor by factor, so extents whose
 * product would overflow are refused too.  All calls share the array and it
 * keeps the last call's
 * contents (each call clears what must start at zero): calls that overlap on
 * the GPU (on different streams, or from different host threads) race and
 * must be ordered by the caller.  No cudaMalloc, cudaFree or allocating
 * library routine is called.                                               */
fsi_status fsi_locate_noalloc(const fsi_grid *grid, int64_t m, const double *X, int32_t *elem,
                              double *xi, int32_t *cell_start, int32_t *perm,
                              int64_t *n_outside, int strict, int device, void *cuda_stream);

/* Interface scaling field of Sec. 2.1: tau_M's bracket is multiplied by s,
 * s >> 1 in an O(h) neighbourhood of the fluid-solid interface and 1
 * elsewhere, defined at the fluid nodes and interpolated like the pressure
 * (Q1), which gives a smooth transition over one element.  The paper fixes no
 * band width; here the band is every cell holding a solid point, dilated by
 * `layers` cells in each direction (clipped at the grid), and
 * s [n] (FP64 device, overwritten) = s_band on every node of a band cell, 1
 * elsewhere.  cell_start [E+1] is fsi_locate's cell table of the points.
 * Pass s as fsi_stage's s (or fsi_step_state.s) on a mesh created with
 * has_s != 0.  s_band > 0 and finite; 0 <= layers <= 64.                  */
fsi_status fsi_interface_scaling(fsi_mesh *mesh, const int32_t *cell_start, double s_band,
                                 int32_t layers, double *s);

/* Interpolation of the fluid velocity to the solid points, u = C^T V
 * (Eq. nodal_solid_velo): u_B = sum_A N_A(xi_B) V_A over the 8 nodes of
 * element elem[B], velocity slots only.  xi [m][3] and U [n][4] and u [m][3]
 * are in `prec` (FSI_F64, FSI_F32 or FSI_DF64 on double arrays); elem [m]
 * int32 from fsi_locate.  Outside points (elem < 0)
 * get u = 0; so do points whose elem is >= E (never produced by
 * fsi_locate), which are never dereferenced.                               */
fsi_status fsi_dlm_interp(fsi_mesh *mesh, fsi_prec prec, int64_t m, const int32_t *elem,
                          const void *xi, const void *U, void *u);

/* Spreading with the FSI constraint matrix C_AB = N_A(xi_B) I
 * (Eq. fsi_constraint_matrix): F_A += sum_B w_B N_A(xi_B) lambda_B into the
 * momentum slots 0..2 of F [n][4]; slot 3 is neither read nor written.
 * accumulate == 0 overwrites slots 0..2 instead of adding.  lam [m][3],
 * w [m] (NULL: w_B = 1), xi [m][3] and F are in `prec` (FP64 for FSI_DF64,
 * which computes in double-float on FP32 units to about 2^-44 relative).
 * elem, cell_start and perm are the outputs of fsi_locate for the same points.  No atomic
 * operation is used and the result is deterministic: each cell's corner sums
 * are formed over its points in perm order with a fixed reduction tree (in
 * mesh scratch), then each node adds the sums of its (up to) 8 cells in a
 * fixed order.                                                            */
fsi_status fsi_dlm_spread(fsi_mesh *mesh, fsi_prec prec, int64_t m, const int32_t *elem,
                          const void *xi, const int32_t *cell_start, const int32_t *perm,
                          const void *lam, const void *w, void *F, int accumulate);

/* Mapped (curvilinear) structured background grid: X [n][3] FP64 device
 * array of node coordinates in the mesh's node numbering (copied), NULL to
 * return to the uniform grid.  Every element must map the parent cube with a
 * positive Jacobian.  With coordinates the VMS operators take the geometry of
 * each Gauss point from the trilinear map (dx/dxi, det, the full metric
 * G_ij = sum_k dxi_k/dx_i dxi_k/dx_j of Sec. 2.1, gradients through J^-T),
 * and fsi_locate finds elements by a bounded walk with Newton inversion of the
 * trilinear map (started in the element the nominal uniform box gives; at
 * most Nx + Ny + Nz + 8 elements, 30 Newton iterations each; a point counts
 * as inside when |xi_k| <= 1 + 1e-10).  Interpolation and spreading only
 * need (elem, xi) and work unchanged.  The nominal N, x0, h of the mesh stay
 * in use for the walk's start and the Schur preconditioner's geometric
 * multigrid (an approximation there; fsi_pressure_use_amg assembles the
 * pressure operator from the coordinates instead).  Synchronises the mesh stream.  The
 * geometry of the Gauss points (J^-1, G, G:G, 1/tr G, det J: 18 values per
 * point) is computed once per compute type, on the first residual or
 * Jacobian apply in it, into a table kept with the mesh (E x 144 values:
 * 8 bytes each for FSI_F64 and FSI_DF64, 4 for FSI_F32) and dropped by the
 * next call of this function; that first apply allocates, so it must not run
 * inside a stream capture (FSI_ERR_ARG then; FSI_ERR_OOM if the table does
 * not fit).                                                                */
fsi_status fsi_mesh_set_coordinates(fsi_mesh *mesh, const double *X);

/* ----------------------------------------------------------------------- */
/* Unstructured tetrahedral background meshes: linear P1-P1 tetrahedra, the  */
/* element family of the paper's valve fluid mesh (Sec. 4), with the same    */
/* VMS weak form (Sec. 2.1), linearisation (Sec. 2.4) and coupling operators */
/* (Sec. 2.3) as the structured grid.                                        */
/*                                                                          */
/* Discretisation: reference tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1),    */
/* N_0 = 1 - xi_1 - xi_2 - xi_3, N_k = xi_k; J = [x1-x0, x2-x0, x3-x0];       */
/* G = J^-T J^-1 (the metric of Sec. 2.1 with this parent domain); the      */
/* symmetric 4-point quadrature rule of degree 2, weight |det J|/24 each.    */
/* Elements may have either orientation.                                     */
/* ----------------------------------------------------------------------- */
typedef struct fsi_tetmesh fsi_tetmesh;

/* Build a tetrahedral mesh on `device`, ordered on `cuda_stream`: X [n][3]
 * FP64 node coordinates and tets [E][4] int32 node numbers, both device
 * arrays (copied; the caller keeps ownership).  Builds the node -> element
 * slot lists of the atomic-free assembly and a uniform bucket grid for point
 * location (host work proportional to n + E); synchronises the stream.
 * FSI_ERR_ARG for bad sizes, node numbers out of range, non-finite
 * coordinates or invalid physics; FSI_ERR_OOM if device memory runs out.  */
fsi_status fsi_tetmesh_create(int64_t n_nodes, const double *X, int64_t n_tets,
                              const int32_t *tets, const fsi_physics *phys, int device,
                              void *cuda_stream, fsi_tetmesh **out);
void fsi_tetmesh_destroy(fsi_tetmesh *mesh);

/* The implicit step on a tetrahedral mesh: an fsi_mesh handle backed by a
 * tetrahedral mesh (same arguments as fsi_tetmesh_create).  On it
 * fsi_residual, fsi_jacobian_apply, fsi_stage, fsi_advance_history,
 * fsi_locate (xi = barycentric lam), fsi_dlm_interp, fsi_dlm_spread,
 * fsi_coupled_residual, fsi_coupled_jacobian_apply, fsi_block_diagonal and
 * fsi_newton_step act as on the structured grid (cell_start has n_tets + 1
 * entries).  The nodal diagonal blocks are probed with a distance-2 node
 * colouring built at creation (no two nodes of one element share a colour);
 * fsi_newton_step takes either preconditioner (the Schur one with an
 * algebraic multigrid for the pressure; see fsi_pressure_vcycle).  The
 * interface band, mapped coordinates, brick shapes, the
 * learned guess (stencil features) and the batched ensemble need a
 * structured grid and return FSI_ERR_ARG on this handle.                   */
fsi_status fsi_mesh_create_tet(int64_t n_nodes, const double *X, int64_t n_tets,
                               const int32_t *tets, const fsi_physics *phys, int device,
                               void *cuda_stream, fsi_mesh **out);

/* VMS residual and Jacobian apply on the tetrahedral mesh: the same
 * arguments, layouts and precisions as fsi_residual / fsi_jacobian_apply
 * (U, A, f, x, R, Jx [n][4] device arrays; f may be NULL).  Deterministic.
 * The first call of each compute type builds that type's per-element
 * geometry table (J^-1, G, the weight: 18 values per element) on the mesh's
 * stream and keeps it with the mesh; it allocates, so that first call must
 * not be made while the stream is being captured into a CUDA graph
 * (FSI_ERR_ARG then).  FSI_ERR_OOM if the table cannot be allocated.      */
fsi_status fsi_tet_residual(fsi_tetmesh *mesh, fsi_prec prec, const void *U, const void *A,
                            const void *f, void *R);
fsi_status fsi_tet_jacobian_apply(fsi_tetmesh *mesh, fsi_prec prec, const void *U,
                                  const void *A, const void *f, const void *x, void *Jx);

/* Point location (Sec. 3, Algorithm 1): for each of the m points P [m][3]
 * (FP64 device array) the element elem [m] and the barycentric coordinates
 * lam [m][3] = (lam_1, lam_2, lam_3) (lam_0 = 1 - their sum).  A point
 * belongs to the lowest-numbered element whose four coordinates, computed in
 * FP64 in the order e_k = x_k - x_0, d = P - x_0, D = e1.(e2 x e3),
 * lam_1 = d.(e2 x e3)/D, lam_2 = e1.(d x e3)/D, lam_3 = e1.(e2 x d)/D,
 * lam_0 = ((1 - lam_1) - lam_2) - lam_3, are all >= -1e-12; others get
 * elem = -1, lam = 0.  cell_start [E+1] / perm [m] (both or neither; perm
 * may be NULL when m = 0) receive the element -> points table (stable,
 * outside points last).  n_outside
 * (host, may be NULL) synchronises the stream.                             */
fsi_status fsi_tet_locate(fsi_tetmesh *mesh, int64_t m, const double *P, int32_t *elem,
                          double *lam, int32_t *cell_start, int32_t *perm, int64_t *n_outside);

/* Interpolation u = C^T U (Eq. nodal_solid_velo) and spreading F = C w lambda
 * (Eq. fsi_constraint_matrix) with the barycentric shape functions; the same
 * arguments, precisions and semantics as fsi_dlm_interp / fsi_dlm_spread
 * (lam in the working precision, FP64 for FSI_DF64).                       */
fsi_status fsi_tet_interp(fsi_tetmesh *mesh, fsi_prec prec, int64_t m, const int32_t *elem,
                          const void *lam, const void *U, void *u);
fsi_status fsi_tet_spread(fsi_tetmesh *mesh, fsi_prec prec, int64_t m, const int32_t *elem,
                          const void *lam, const int32_t *cell_start, const int32_t *perm,
                          const void *lamv, const void *w, void *F, int accumulate);

/* Self-test of the bounded waits in the tensor-core kernels (no counterpart
 * in the paper): one thread waits, with the same wait loop the kernels use,
 * on an mbarrier whose expected arrival never comes.  The wait gives up after
 * its poll limit (a few seconds at most), the kernel raises its error flag and
 * returns, and the context stays usable.  *timed_out = 1 when that happened,
 * *seconds = the kernel's time.  Synchronises the device.                   */
fsi_status fsi_wait_selftest(int device, int *timed_out, double *seconds);

/* ----------------------------------------------------------------------- */
/* One implicit step: the reduced FSI system of Sec. 2.4.                    */

/* The state of one time step.  All arrays are DEVICE pointers, FP64.
 * The unknown y = (Vdot_{n+1}, P_{n+1}) [n][4]; Vn = (V_n, -) and
 * An = (Vdot_n, -) [n][4] are the history (slot 4 ignored); s [n] and
 * f [n][4] are optional (NULL).  Dirichlet rows: mask [n][4] (uint8, nonzero
 * = Dirichlet) with prescribed values yD [n][4]; both NULL for none.
 * Immersed solid (may have m = 0): the m points located at the start of the
 * step by fsi_locate (elem, xi [m][3] FP64, cell_start, perm), weights w [m]
 * (NULL: 1).  The paper's solid residual R^s needs FEBio constitutive code;
 * this library uses a point-mass stand-in per point B:
 *   r^s_B = drho_s (a_B - g_s) + k_s dx_B,  a_B = (C^T Vdot_{n+1})_B,
 *   dx_B = dt (C^T V_{n+1})_B,
 * spread with the point weights: R^{f,m} += C W r^s, so that the solid block
 * of the reduced Jacobian is C W (drho_s + k_s gamma dt^2) C^T.            */
typedef struct fsi_solid fsi_solid;

typedef struct {
    double *y;
    const double *Vn, *An, *s, *f;
    const uint8_t *mask;
    const double *yD;
    int64_t m;
    const int32_t *elem, *cell_start, *perm;
    const double *xi, *w;
    double drho_s, k_s;
    double g_s[3];
    /* hyperelastic immersed solid (fsi_solid_create) instead of the
     * point-mass stand-in, or NULL.  When set, the m points are the solid's
     * nodes located at X + us (m = its node count; w, drho_s, k_s are
     * ignored; g_s is the body force f of Sec. 2.2), and us, vs, as [m][3]
     * FP64 are its displacement, velocity and acceleration at t_n.          */
    fsi_solid *body;
    const double *us, *vs, *as;
} fsi_step_state;

/* Full residual of the reduced system (Sec. 2.4) at st->y:
 * R = [R^{f,m} + C W r^s ; R^{f,c}] with Dirichlet rows replaced by y - yD.
 * R [n][4] FP64 device, overwritten.  prec = FSI_F64 computes in native FP64,
 * FSI_DF64 the VMS residual, interpolation and spreading in double-float
 * (FP64-accurate to ~1e-14 relative, several times faster on GB300); the
 * stage values and the solid force are FP64 in both.                       */
fsi_status fsi_coupled_residual(fsi_mesh *mesh, fsi_prec prec, const fsi_step_state *st,
                                double *R);

/* Jacobian-vector product of fsi_coupled_residual at st->y in `prec`:
 * Jx = J_f x + C W (drho_s + k_s gamma dt^2) C^T x_v, with Dirichlet rows
 * of Jx equal to those of x.  x and Jx [n][4] are in `prec` (the
 * linearisation point is converted to `prec` internally).                  */
fsi_status fsi_coupled_jacobian_apply(fsi_mesh *mesh, fsi_prec prec, const fsi_step_state *st,
                                      const void *x, void *Jx);

/* Nodal 4x4 diagonal blocks of the coupled Jacobian at st->y, by probing
 * with the 8 node colours x 4 components (nodes of one colour share no
 * element or cell, so each probe returns exact diagonal blocks):
 * blocks [n][4][4] in `prec`, row-major (row = residual slot, column =
 * unknown slot).  Dirichlet rows are unit rows.                            */
fsi_status fsi_block_diagonal(fsi_mesh *mesh, fsi_prec prec, const fsi_step_state *st,
                              void *blocks);

/* Newton on the reduced system (Sec. 2.4) from st->y (the predictor; on
 * return the iterate that met the tolerance, or the last one).  Each
 * iteration: FP64 residual; right-preconditioned restarted GMRES on
 * J dy = -R (preconditioner per opts.precond); y += dy in FP64.
 *   mixed = 0: every step in FP64 (the plain method);
 *   mixed = 1: Krylov vectors, Jacobian applies and preconditioner in FP32;
 *              the residual, the Gram-Schmidt dot products and norms (FP64
 *              accumulation), the Hessenberg least-squares problem and the
 *              update stay FP64 (defect correction).
 * Stops when ||R(y_k)||_2 <= newton_rtol * r_ref, r_ref = ||R(y_0)||_2 when
 * opts.r_ref <= 0.  GMRES at iteration k stops at the relative tolerance
 * max(krylov_rtol, min(0.5, 0.5 target / ||R(y_k)||)) (no oversolving near
 * the target).  Synchronises.  Returns FSI_ERR_NOCONV when max_newton
 * iterations did not reach the tolerance, FSI_ERR_NAN on a non-finite norm;
 * the report is filled in every case.  Workspace is kept in the mesh.      */
typedef struct {
    int32_t mixed;
    int32_t restart;       /* GMRES restart length, 1..200 (e.g. 50)          */
    int32_t max_newton;    /* Newton iterations at most                       */
    int32_t max_krylov;    /* Krylov iterations per Newton iteration at most  */
    double newton_rtol;    /* e.g. 1e-8                                        */
    double krylov_rtol;    /* inner relative tolerance, e.g. 1e-3              */
    double r_ref;          /* > 0: reference norm of the stopping test         */
    int32_t precond_every; /* rebuild the preconditioner every k Newton
                              iterations (0: build once per call, at y_0)     */
    int32_t precond;       /* 0: nodal 4x4 block-Jacobi; 1: block-diagonal
                              Schur-complement preconditioner (3x3 velocity
                              blocks, pressure Schur complement approximated
                              by sigma (K + kappa M) and inverted by one
                              multigrid V-cycle: geometric on the structured
                              grid, algebraic on a tetrahedral mesh; see
                              fsi_pressure_vcycle)                            */
    int32_t residual_prec; /* FSI_F64 or FSI_DF64: arithmetic of the Newton
                              residual (see fsi_coupled_residual)             */
    int32_t reserved;
    const double *R0;      /* NULL, or R(y_0) [n][4] FP64 on the device,
                              computed by the caller in residual_prec for
                              this state (fsi_coupled_residual, e.g. the
                              judge's residual fsi_mlp_guess leaves in its
                              work array): the first residual evaluation is
                              skipped.  Ignored (R(y_0) evaluated) when the
                              state carries a hyperelastic body, whose stage
                              values come out of the residual.  Read only.   */
} fsi_newton_opts;

typedef struct {
    int32_t newton_iters;  /* Newton corrections applied                      */
    int32_t krylov_iters;  /* GMRES iterations summed over Newton iterations   */
    double r0;             /* ||R(y_0)||_2                                     */
    double r_final;        /* ||R(y)||_2 of the returned y                     */
    double r_ref;          /* reference norm used by the stopping test         */
    double seconds;        /* wall time of the call                            */
    int32_t converged;
    int32_t precond_builds;
} fsi_newton_report;

fsi_status fsi_newton_step(fsi_mesh *mesh, const fsi_newton_opts *opts, const fsi_step_state *st,
                           fsi_newton_report *report);


/* ----------------------------------------------------------------------- */
/* Immersed hyperelastic solid (Sec. 2.2, Eq. solid_weak_form) on a Q1
 * hexahedral solid mesh.  Nodal residual
 *   R^s_a = sum_g N_a (rho_s - rho_f)(uddot(g) - f) detJ0
 *         + sum_g P(F) grad_X N_a detJ0
 *         - sum_g 2 mu_f D grad_x N_a J detJ0
 * (2x2x2 Gauss points in the reference configuration; compressible
 * neo-Hookean P = mu_s (F - F^-T) + lambda_s ln J F^-T; D the symmetric
 * gradient of the solid's velocity field on the configuration X + u_n at the
 * start of the step; rho_f and mu_f are the mesh's fluid properties).  The
 * paper leaves the material and the evaluation of the artificial-fluid term
 * open; these are this library's choices.  Time stepping is generalized-alpha
 * with Newmark beta = (1 + alpha_m - alpha_f)^2 / 4: the residual is taken
 * at uddot_{n+alpha_m}, v_{n+alpha_f}, u_{n+alpha_f}, functions of
 * uddot_{n+1} = C^T Vdot_{n+1}; in fsi_newton_step the reduced system gets
 * R^{f,m} += C R^s and J += C dR^s/duddot_{n+1} C^T (Sec. 2.4).
 *
 * X [n_nodes][3] (reference coordinates) and conn [n_elems][8] (corner a =
 * ax + 2 ay + 4 az of the element's trilinear map, positive Jacobian) are
 * device arrays, copied.  All nodal arrays below are [n_nodes][3] FP64 device
 * arrays unless a precision is given.  Calls run on the mesh's stream.      */
fsi_status fsi_solid_create(fsi_mesh *mesh, int64_t n_nodes, int64_t n_elems, const double *X,
                            const int32_t *conn, double rho_s, double mu_s, double lambda_s,
                            fsi_solid **out);
void fsi_solid_destroy(fsi_solid *body);
/* R [n][3] = R^s at the stage values (u_af, v_af, a_am), viscous term on
 * X + u_n; g [3] the body force f (NULL: 0).                                */
fsi_status fsi_solid_residual(fsi_solid *body, const double *u_af, const double *v_af,
                              const double *a_am, const double *u_n, const double *g, double *R);
/* Jx = dR^s/duddot_{n+1} x = alpha_m M x + alpha_f beta dt^2 K(u_af) x
 *      - alpha_f gamma dt K_visc(u_n) x, with u_af, x, Jx in `prec`.         */
fsi_status fsi_solid_tangent_apply(fsi_solid *body, fsi_prec prec, const void *u_af,
                                   const double *u_n, const void *x, void *Jx);
/* stage values from uddot_{n+1} and the history (u, v, a) at t_n           */
fsi_status fsi_solid_stage(fsi_solid *body, const double *u, const double *v, const double *a,
                           const double *a_next, double *u_af, double *v_af, double *a_am);
/* history advance (u, v, a) <- (u_{n+1}, v_{n+1}, uddot_{n+1}), in place     */
fsi_status fsi_solid_advance(fsi_solid *body, double *u, double *v, double *a,
                             const double *a_next);
/* current node positions x = X + u (to locate the nodes for the next step) */
fsi_status fsi_solid_positions(fsi_solid *body, const double *u, double *x);
/* ----------------------------------------------------------------------- */
/* Pressure block of the Schur-complement preconditioner (opts.precond = 1;
 * Sec. 2.4 solves the reduced system with block preconditioners built from
 * its sub-matrices).  With the fluid blocks [[A, B], [C, D]] (A = dR^{f,m}/dVdot
 * mass-dominated, B gradient, C = c_v x divergence + PSPG, D PSPG), the
 * pressure Schur complement D - C A^{-1} B is approximated by sigma (K + kappa M):
 * K, M the Q1 stiffness and mass matrices of the pressure space on the mesh
 * grid, sigma = alpha_f gamma dt / (alpha_m rho), kappa = (pi / (2 L))^2 with L
 * the largest grid extent.  Its inverse is replaced by one V-cycle over the
 * levels: the mesh grid, then every other node while all N_d are even and the
 * level has more than 125 nodes; trilinear prolongation P, restriction P^T;
 * Chebyshev smoothing of degree 2 (pre and post) on D^{-1}(K + kappa M) over
 * [hi/4, hi] (hi = 1.1 x the largest symbol-to-diagonal ratio of the modes
 * theta_d in {0, pi}); a dense inverse on a coarsest level of <= 1000 nodes,
 * else Chebyshev of degree 8 over [hi/30, hi].  The paper fixes none of these
 * choices; the V-cycle is a fixed symmetric linear operator.
 *
 * On a face of the box where the velocity is free (a traction-free outflow)
 * the true Schur complement acts like a Dirichlet problem for the pressure:
 * the nodes of "eliminated" faces keep only their diagonal entry and drop
 * out of every other row, on every level, and the restricted right-hand side
 * is zeroed there.  fsi_newton_step picks the faces from its Dirichlet mask:
 * a face is eliminated when more than half of the nodes inside it (off its
 * edges; all its nodes if none is inside) have all three velocity
 * components free.
 *
 * Vectors are scalar nodal fields [n_l] of the level (lexicographic, x
 * fastest) in `prec` (FSI_F64 or FSI_F32), device pointers owned by the
 * caller.  Level 0 is the mesh grid.  The hierarchy is built on first use
 * and kept in the mesh.  Stream-ordered on the mesh stream.
 *
 * On an fsi_mesh backed by a tetrahedral mesh (fsi_mesh_create_tet) the same
 * entry points act on K + kappa M of the P1 pressure space (element
 * matrices K_ab = V grad l_a . grad l_b, M_ab = V (1 + delta_ab) / 20; L the
 * largest extent of the bounding box), and the levels are those of a
 * smoothed-aggregation algebraic multigrid built on the host in FP64 (one
 * synchronisation) on first use and whenever the elimination set changes:
 * strong neighbours |a_ij| >= 0.08 sqrt(a_ii a_jj); greedy aggregation in
 * node order; P = (I - 4/(3 rho) D^-1 A) P0 with P0 the aggregate indicator
 * and rho the spectral radius of D^-1 A (30 power iterations, at most the
 * Gershgorin bound); R = P^T, Galerkin coarse operators R A P; levels until
 * <= 600 unknowns (dense inverse) or the coarsening stalls; Chebyshev of
 * degree 2 over [hi/10, hi], hi = 1.1 rho.  Vectors are in node order.
 * Eliminated nodes are given per node (fsi_pressure_set_eliminated); none
 * by default.  fsi_newton_step eliminates the nodes on the mesh boundary
 * whose three velocity components are free and the nodes whose pressure is
 * fixed.  fsi_pressure_levels and fsi_pressure_set_faces are for the
 * geometric multigrid of the structured grid only (FSI_ERR_ARG here).
 *
 * A structured grid takes the same algebraic multigrid after
 * fsi_pressure_use_amg(mesh, 1): K + kappa M is then assembled from the Q1
 * element matrices of the grid's hexahedra (corner a of element (i, j, k) at
 * node (i + (a&1), j + ((a>>1)&1), k + ((a>>2)&1)); eight Gauss points
 * +-1/sqrt(3), the quadrature of the VMS operators: exact on affine maps,
 * and on a trilinear map K still annihilates linear fields at interior
 * nodes) at the mapped node
 * coordinates when fsi_mesh_set_coordinates gave some, else on the uniform
 * grid (where it equals the geometric multigrid's level-0 operator); L is
 * the largest extent of the nodes' bounding box; boundary nodes are those on
 * the box's faces; the strength threshold is 0.02 (the Q1 stiffness couples
 * a near-cubic element's edge and corner neighbours by 1/16 and 1/32 of the
 * diagonal).  This is the pressure operator assembled on the mapped
 * geometry, where the geometric multigrid uses the nominal uniform one.     */
/* number of levels and the unknowns per level n[l] ([16] or NULL); either
 * mesh kind */
fsi_status fsi_pressure_level_sizes(fsi_mesh *mesh, int32_t *n_levels, int64_t *n);
/* select the pressure block of a structured grid: on != 0 the algebraic
 * multigrid from the assembled element matrices, 0 the geometric multigrid
 * (the default).  Synchronises the mesh stream when the choice changes; the
 * hierarchy is built on first use and dropped (with its elimination set) by
 * a change of choice or of coordinates.  On a tetrahedral mesh on = 0 is
 * FSI_ERR_ARG and on != 0 does nothing.                                     */
fsi_status fsi_pressure_use_amg(fsi_mesh *mesh, int32_t on);
/* algebraic multigrid only (tetrahedral mesh, or fsi_pressure_use_amg):
 * eliminated[n] device flags (nonzero = eliminated), NULL = none.
 * Synchronises the mesh stream; rebuilds the hierarchy when the set changes.
 * FSI_ERR_ARG with the geometric multigrid.                                 */
fsi_status fsi_pressure_set_eliminated(fsi_mesh *mesh, const uint8_t *eliminated);
/* faces[6] (x0, x1, y0, y1, z0, z1), nonzero = eliminated; none by default.
 * Synchronises the mesh stream when the set changes (the coarse inverse is
 * rebuilt).                                                                */
fsi_status fsi_pressure_set_faces(fsi_mesh *mesh, const int32_t *faces);
fsi_status fsi_pressure_levels(fsi_mesh *mesh, int32_t *n_levels, int32_t *N /* [16][3] or NULL */);
/* y = (K + kappa M) x on level `level` */
fsi_status fsi_pressure_apply(fsi_mesh *mesh, fsi_prec prec, int32_t level, const void *x, void *y);
/* b (level+1) = P^T r (level) */
fsi_status fsi_pressure_restrict(fsi_mesh *mesh, fsi_prec prec, int32_t level, const void *r,
                                 void *b);
/* x (level) += P xc (level+1) */
fsi_status fsi_pressure_prolong_add(fsi_mesh *mesh, fsi_prec prec, int32_t level, const void *xc,
                                    void *x);
/* `degree` Chebyshev steps on level `level` over [hi/4, hi] ([hi/10, hi] on a
 * tetrahedral mesh) for (K + kappa M) x = b,
 * from x = 0 (from_zero != 0; x is overwritten) or from the given x.  Uses the
 * level's scratch direction vector. */
fsi_status fsi_pressure_smooth(fsi_mesh *mesh, fsi_prec prec, int32_t level, int32_t degree,
                               const void *b, void *x, int32_t from_zero);
/* x = V(b) ~ (K + kappa M)^{-1} b on the mesh grid (b, x: [n], not aliased). */
fsi_status fsi_pressure_vcycle(fsi_mesh *mesh, fsi_prec prec, const void *b, void *x);

/* ----------------------------------------------------------------------- */
/* Learned initial guess (an extension; the paper has no counterpart).      */
/* A 112 -> 256 -> 256 -> 4 ReLU network predicts, per node, the correction c
 * to the extrapolated increment e = 2 d_{n-1} - d_{n-2} (d_k = y_{k+1} - y_k)
 * so that the Newton predictor is y^(0) = y_n + e + c.  Inputs per node: the
 * 27-node stencil (offsets -1..1 per axis, x fastest, zero outside the grid)
 * of (V_n velocity, P_n pressure) = 108 values, then e (4); each normalised
 * as (x - in_mean) / in_std.  Outputs o are de-normalised as
 * c = out_mean + out_std * o.
 * Parameters: one FP32 device vector of fsi_mlp_num_params() values laid out
 * W1 [112][256], b1 [256], W2 [256][256], b2 [256], W3 [256][4], b3 [4]
 * (row = input unit).  The GEMMs run on the 5th-generation tensor cores
 * (tcgen05, TMEM accumulators) with BF16 operands and FP32 accumulation; the
 * weight-gradient GEMMs sum split-K partial tiles in a fixed order, so
 * results are deterministic.  Loss = (1/B) sum_rows 1/2 |o - t|^2.
 * forward, loss_grad, adam and predict are asynchronous on their streams.
 * The tensor-core kernels bound every wait; a wait that runs out (which only
 * a stuck tensor-core pipeline would cause) leaves an error flag on the
 * handle that fsi_mlp_check and fsi_mlp_guess report as FSI_ERR_TIMEOUT.   */
typedef struct fsi_mlp fsi_mlp;

/* Handle with activation scratch for batches of up to max_batch rows. */
fsi_status fsi_mlp_create(int device, void *cuda_stream, int64_t max_batch, fsi_mlp **out);
void fsi_mlp_destroy(fsi_mlp *mlp);
int64_t fsi_mlp_num_params(void);

/* out [B][4] = network(X [B][112]) (normalised units). */
fsi_status fsi_mlp_forward(fsi_mlp *mlp, const float *params, const float *X, int64_t B,
                           float *out);

/* loss (device scalar) and grad [num_params] of the batch (X [B][112], T [B][4]). */
fsi_status fsi_mlp_loss_grad(fsi_mlp *mlp, const float *params, const float *X, const float *T,
                             int64_t B, float *loss, float *grad);

/* One Adam step (bias-corrected; step counts from 1) on params, in place. */
fsi_status fsi_mlp_adam(fsi_mlp *mlp, float *params, const float *grad, float *m, float *v,
                        int step, float lr, float beta1, float beta2, float eps);

/* Normalised features X [k][112] of the nodes idx [k] (all n nodes when idx
 * is NULL) from Vn [n][4] (velocity slots), y [n][4] (pressure slot) and the
 * last two increments d1, d2 [n][4]; FP64 inputs, FP32 output.            */
fsi_status fsi_mlp_features(fsi_mesh *mesh, const double *Vn, const double *y, const double *d1,
                            const double *d2, const int32_t *idx, int64_t k,
                            const float *in_mean, const float *in_std, float *X);

/* Reports and clears the handle's tensor-core error flag (see above):
 * FSI_ERR_TIMEOUT if a wait of an earlier call ran out, else FSI_OK.
 * Synchronises the device.                                                 */
fsi_status fsi_mlp_check(fsi_mlp *mlp);

/* Newton predictor y0 [n][4] = y + e + c for every node, on the mesh's
 * stream, by one fused tensor-core kernel (features, three layers,
 * predictor).  Asynchronous.                                               */
fsi_status fsi_mlp_predict(fsi_mlp *mlp, fsi_mesh *mesh, const float *params,
                           const float *in_mean, const float *in_std, const float *out_mean,
                           const float *out_std, const double *Vn, const double *y,
                           const double *d1, const double *d2, double *y0);

/* The FP64 residual judges the network.  With d1, d2 the last two
 * increments, e = 2 d1 - d2 their linear extrapolant and c = y_ml - y_n - e
 * the network's correction (fsi_mlp_predict), the predictor is the best
 * member of the family
 *     y = y_fb + x1 d1 + x2 d2 + x3 c
 * around the fallback y_fb (fallback 0: y_n, the zero increment; 1: y_n + e),
 * all Dirichlet rows (st->mask) held at st->yD: the coefficients minimise
 * |R(y_fb) + J (x1 d1 + x2 d2 + x3 c)|, R the coupled
 * residual of y_fb (its VMS part in FP32 from the FP32 linearisation, the
 * coupling and the Dirichlet rows double-float: the fit needs R far better
 * than the reduction a predictor brings, not to FP64) and J its Jacobian at
 * y_fb applied in FP32 (fsi_coupled_jacobian_apply; R is close to linear in y
 * over a predictor's error), by the 3 x 3 normal equations in FP64 (a
 * direction that adds nothing is dropped).  The family holds both fallbacks
 * (the zero increment and e) and the network's own predictor, so the fit is
 * at least as good as each of them in the linear model.  The candidate's
 * residual is then evaluated in judge_prec, and st->y keeps the candidate if
 * its norm is below the fallback's (r_fallback), else y_fb.  Cost: the
 * network, one FP32 linearisation with the FP32 residual and three FP32
 * Jacobian applies, and the candidate's residual in judge_prec (which a
 * Newton step can take as its first, fsi_newton_opts.R0; when the fallback
 * is kept, its residual in judge_prec is evaluated instead).  judge_prec:
 * FSI_F64 or FSI_DF64.  work: caller-owned FP64 device array [5][n][4]; on
 * return work[0..n) x 4 holds R(st->y) in judge_prec, for
 * fsi_newton_opts.R0.
 * yn [n][4] is y_n (must not alias st->y).  Synchronises; a tensor-core wait
 * that ran out in this or an earlier call of the handle is FSI_ERR_TIMEOUT. */
typedef struct {
    double r_fallback;   /* ||R(y_fb)||_2, the fit's residual (VMS part FP32)      */
    double r_learned;    /* the linear model's ||R|| at the network's own predictor */
    double r_combined;   /* ||R(y_c)||_2 of the fitted candidate, judge_prec         */
    double c_d1, c_d2, c_net;  /* x1, x2, x3                                      */
    int32_t used;        /* 0 fallback, 2 fitted candidate                           */
    int32_t reserved;
    double r_history_fit; /* the linear model's ||R|| at the best y_fb + x1 d1 +
                             x2 d2 alone (the same fit without the network's
                             direction: what the network adds is the gap to
                             r_combined)                                       */
} fsi_guess_report;

fsi_status fsi_mlp_guess(fsi_mlp *mlp, fsi_mesh *mesh, const float *params, const float *in_mean,
                         const float *in_std, const float *out_mean, const float *out_std,
                         const fsi_step_state *st, const double *yn, const double *d1,
                         const double *d2, int fallback, fsi_prec judge_prec, double *work,
                         fsi_guess_report *rep);

/* ----------------------------------------------------------------------- */
/* Batched ensemble (an extension; the paper has no counterpart).           */
/* Many independent instances (each its own mesh: grid, physics) of uneven
 * size.  One item per instance: device arrays in the batch's precision,
 * contiguous, owned by the caller and kept valid (same pointers) for the
 * batch's lifetime: U, A, f (or NULL), x, R, Jx [n_i][4]; points (m may be
 * 0, m < 2^31): elem [m], cell_start [E_i+1], perm [m], xi [m][3],
 * lam [m][3], w [m] (or NULL), u [m][3]; spreading writes F [n_i][4]
 * (slots 0..2, overwrite).
 * X [m][3] (FP64) are the instance's raw solid points, or NULL.  With X the
 * step locates them itself (Sec. 3, Algorithm 1's point search; the rule of
 * fsi_locate): elem, xi, cell_start and perm are OUTPUTS of every step,
 * written bit for bit as fsi_locate writes them (xi rounded to FP32 in an
 * FP32 batch), so they must point to writable memory.  Without X they are
 * inputs from an earlier fsi_locate.
 * One batched step = for every instance (locate X), R = residual(U, A, f),
 * Jx = J(U, A, f) x, u = C^T U, F = C lambda.                              */
typedef struct {
    const void *U, *A, *f, *x;
    void *R, *Jx;
    int64_t m;
    const int32_t *elem, *cell_start, *perm;
    const void *xi, *lam, *w;
    void *u, *F;
    const double *X;
} fsi_batch_item;

typedef struct fsi_batch fsi_batch;

enum {
    FSI_BATCH_PER_INSTANCE = 0, /* the single-mesh entry points, instance by instance */
    FSI_BATCH_PERSISTENT = 1,   /* persistent grids over all instances' work items      */
    FSI_BATCH_GRAPH = 2         /* the persistent step captured once in a CUDA graph and
                                   replayed (needs a non-default stream)                */
};

/* Build a batch (descriptors, prefix sums and its own scratch) on `cuda_stream`.
 * All meshes must be on one device and uniform (no fsi_mesh_set_coordinates;
 * FSI_ERR_ARG otherwise).  The batch uses one brick shape for all instances
 * (default 8x8x4; see fsi_batch_autotune).                                 */
fsi_status fsi_batch_create(fsi_mesh *const *meshes, const fsi_batch_item *items, int count,
                            fsi_prec prec, void *cuda_stream, fsi_batch **out);
void fsi_batch_destroy(fsi_batch *batch);

/* One batched step in the given mode (results are bitwise identical across
 * modes for a given brick shape).  Asynchronous on the batch's stream.     */
fsi_status fsi_batch_run(fsi_batch *batch, int mode);

/* Seconds per batched step in `mode` (CUDA events, best of reps; synchronises). */
fsi_status fsi_batch_time(fsi_batch *batch, int mode, int reps, double *seconds);

#define FSI_TUNE_MAX_CANDIDATES 64
typedef struct {
    int32_t bx, by, bz, threads, ctas_per_sm;
    int32_t n_candidates;
    double seconds;  /* residual + Jacobian phases of the chosen schedule */
    int32_t cand_bx[FSI_TUNE_MAX_CANDIDATES], cand_by[FSI_TUNE_MAX_CANDIDATES],
        cand_bz[FSI_TUNE_MAX_CANDIDATES], cand_ctas[FSI_TUNE_MAX_CANDIDATES];
    double cand_seconds[FSI_TUNE_MAX_CANDIDATES];
} fsi_tune_report;

/* Autotuner: times every candidate brick shape (elements per CTA along each
 * axis, CTA size) and persistent grid size (CTAs per SM) on this batch's
 * residual + Jacobian phases and keeps the fastest.  When the environment
 * variable FSI_TUNE_CACHE names a file, the choice is appended to it as one
 * JSON object per line.  Synchronises.                                     */
fsi_status fsi_batch_autotune(fsi_batch *batch, int reps, fsi_tune_report *report);

/* Brick schedule of a single mesh for op 0 (residual), 1 (Jacobian) or 2
 * (both fused; twice the shared memory) in compute type
 * `prec` (FSI_F64, FSI_F32 or FSI_DF64, each its own): bx*by*bz elements per CTA of `threads` threads (8 lanes per element;
 * threads a multiple of 32 and at most 256; bx*by*bz*8 >= threads not
 * required).  Scratch grows as needed.                                     */
fsi_status fsi_mesh_set_brick(fsi_mesh *mesh, int op, fsi_prec prec, int bx, int by, int bz,
                              int threads);

/* Autotuner of a single structured mesh: times the VMS residual (op 0),
 * Jacobian apply (op 1) or both fused (op 2, fsi_residual_jacobian_apply) in
 * compute type `prec` on scratch inputs for a fixed
 * set of brick shapes (8x8x4, 8x4x4, 8x8x2, 4x4x4, 4x4x8, 16x4x4 at 256
 * threads; 8x4x4, 4x4x4, 8x4x2, 4x4x2 at 128) and keeps the fastest, as
 * fsi_mesh_set_brick would.  Each compute type (FSI_F64, FSI_F32,
 * FSI_DF64) has its own schedule per operator.  The report's cand_ctas holds each
 * candidate's CTA size, ctas_per_sm is 0; seconds is per launch (brick and
 * gather kernels, mean of reps after one warm-up).  Synchronises; results
 * of later calls do not depend on the schedule's choice beyond rounding
 * order (the element-to-node sums follow the bricks).                      */
fsi_status fsi_mesh_autotune(fsi_mesh *mesh, int op, fsi_prec prec, int reps,
                             fsi_tune_report *report);

/* Measurement helper (the paper has no counterpart): the device's sustained
 * FMA throughput on the CUDA cores in `prec`, in FLOP/s (an FMA counts as 2),
 * from a dependent-chain FMA kernel over all SMs timed with CUDA events
 * (best of 3).  It is the ALU roofline of the VMS operators.  Uses its own
 * stream and a small buffer it allocates and frees; synchronises.          */
fsi_status fsi_measure_fma_peak(int device, fsi_prec prec, double *flops_per_second);

/* Measurement helper (the paper has no counterpart): seconds per call of the
 * Krylov solver's BLAS-1 kernels on vectors of `len` entries (a multiple of
 * 4) in `prec` (FSI_F64, or FSI_F32 as in the mixed mode): the multi-dot of
 * nvec basis vectors with one vector (partial sums and their fixed-order
 * final sums; the reads are nvec + ceil(nvec / 8) vectors), and the
 * multi-update w -= V h over nvec vectors with the fused |w|^2 (nvec + 1
 * reads, 1 write).  1 <= nvec <= 256.  CUDA events over reps calls after one
 * warm-up, on its own stream and buffers, which it allocates and frees;
 * synchronises.                                                            */
fsi_status fsi_measure_blas1(int device, fsi_prec prec, int64_t len, int nvec, int reps,
                             double *dot_seconds, double *axpy_seconds);

/* The Krylov solver's multi-dot by itself (the paper has no counterpart;
 * Sec. 2.4 keeps the Gram-Schmidt dot products in FP64): out[k] = V_k . w
 * for k < nvec, V_k = V + k * ldv, each of `len` entries (len and ldv
 * multiples of 4, V and w 16-byte aligned), in `prec`: FSI_F64 sums in FP64;
 * FSI_F32 forms each product exactly (TwoProd) and sums on the FP32 pipe
 * with a compensated float pair, to the FP64 level (error a few units of
 * 2^-44 of the sum of |V_k[i] w[i]|).  out: FP64 device array [nvec].  The
 * sums follow a fixed grid, so the results are bitwise repeatable.  1 <=
 * nvec <= 256.  Asynchronous on the default stream of `device`.             */
fsi_status fsi_multi_dot(int device, fsi_prec prec, int64_t len, int nvec, const void *V,
                         int64_t ldv, const void *w, double *out);

#ifdef __cplusplus
}
#endif

#endif /* FSI_H */
