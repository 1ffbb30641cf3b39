/*
 * fsi_oracle.c -- plain, slow FP64 CPU oracle for the immersed-FSI hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of
 * bench.py use it.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - Q1 (trilinear) shape functions on the parent cube [-1,1]^3
 *     (first-order Lagrange elements, Sec. 4 intro).
 *   - The VMS-stabilised incompressible Navier-Stokes residual on a uniform
 *     hexahedral background grid: the Galerkin weak form of Eq. (fluid_weak_form)
 *     plus the residual-based VMS terms of Bazilevs et al. 2007 that Sec. 2.1
 *     refers to, with tau_m, tau_c, G from Sec. 2.1 (C_I = 36, C_T = 4).
 *   - The consistent Jacobian-vector product of that residual with respect to
 *     the generalized-alpha unknowns (Sec. 2.4, reduced system), written out
 *     term by term.
 *   - Point location, the interpolation u_A = sum_B N_B(phi(X_A)) v_B of
 *     Eq. (nodal_solid_velo) and the spreading C^lambda lambda with
 *     C_AB = N_A(phi(X_B)) I of Eq. (fsi_constraint_matrix) (Sec. 2.3).
 *   - The same operators on mapped structured grids (node coordinates) and on
 *     unstructured meshes of linear tetrahedra (the element family of the
 *     paper's valve mesh, Sec. 4), with the weak form per quadrature point
 *     shared by all element types (gp_residual, gp_jacobian).
 *
 * Everything is the definition written out: loops over elements, the eight
 * 2x2x2 Gauss points and the eight test nodes; no sum factorisation, no
 * colouring, no blocking.  Element contributions are computed independently
 * (optionally with OpenMP) into element-local buffers and then assembled
 * serially in element order.
 *
 * Layouts: nodes are lexicographic with x fastest, node(i,j,k) =
 * i + (Nx+1)*(j + (Ny+1)*k); elements likewise with Nx, Ny; every nodal field
 * is [n][4] row-major (vx, vy, vz, p) for U, (ax, ay, az, s) for A.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Q1 shape functions.  Local node a = ax + 2*ay + 4*az sits at parent
 * coordinates xi^a_k = 2*a_k - 1; N_a(xi) = 1/8 prod_k (1 + xi_k xi^a_k).   */
void or_shape(const double xi[3], double N[8], double dNdxi[24])
{
    for (int a = 0; a < 8; ++a) {
        double s0 = (a & 1) ? 1.0 : -1.0;
        double s1 = (a & 2) ? 1.0 : -1.0;
        double s2 = (a & 4) ? 1.0 : -1.0;
        double l0 = 1.0 + s0 * xi[0];
        double l1 = 1.0 + s1 * xi[1];
        double l2 = 1.0 + s2 * xi[2];
        N[a] = l0 * l1 * l2 / 8.0;
        dNdxi[3 * a + 0] = s0 * l1 * l2 / 8.0;
        dNdxi[3 * a + 1] = l0 * s1 * l2 / 8.0;
        dNdxi[3 * a + 2] = l0 * l1 * s2 / 8.0;
    }
}

static int64_t node_id(const int N[3], int i, int j, int k)
{
    return (int64_t)i + (int64_t)(N[0] + 1) * ((int64_t)j + (int64_t)(N[1] + 1) * k);
}

/* global node of local node a of element (ex,ey,ez) */
static int64_t elem_node(const int N[3], int ex, int ey, int ez, int a)
{
    return node_id(N, ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1));
}

/* ------------------------------------------------------------------------ */
/* Stabilisation parameters of Sec. 2.1:
 *   tau_m = ( s ( C_T/dt^2 + v.G v + C_I (mu/rho)^2 G:G ) )^(-1/2)
 *   tau_c = ( tau_m tr G )^(-1)
 *   G_ij  = sum_k dxi_k/dx_i dxi_k/dx_j.
 * On the axis-aligned uniform grid dxi_k/dx_k = 2/h_k, so G = diag(4/h_k^2).
 * ct_dt2 is C_T/dt^2 (0 for a steady problem).                               */
static void tau_of_G(const double v[3], double s, const double G[3][3], double rho, double mu,
                     double ct_dt2, double C_I, double out[2])
{
    double trG = 0.0, GG = 0.0, vGv = 0.0;
    for (int i = 0; i < 3; ++i) {
        trG += G[i][i];
        for (int j = 0; j < 3; ++j) {
            GG += G[i][j] * G[i][j];
            vGv += v[i] * G[i][j] * v[j];
        }
    }
    double nu = mu / rho;
    double tau_m = 1.0 / sqrt(s * (ct_dt2 + vGv + C_I * nu * nu * GG));
    out[0] = tau_m;
    out[1] = 1.0 / (tau_m * trG);
}

void or_tau(const double v[3], double s, const double h[3], double rho, double mu,
            double ct_dt2, double C_I, double out[2])
{
    double G[3][3] = {{0}};
    for (int k = 0; k < 3; ++k) G[k][k] = 4.0 / (h[k] * h[k]);
    tau_of_G(v, s, G, rho, mu, ct_dt2, C_I, out);
}

/* Physical parameters passed as an array so that ctypes stays simple:
 * phys[0]=rho, phys[1]=mu, phys[2]=C_T/dt^2, phys[3]=C_I, phys[4]=has_s.   */
typedef struct {
    double rho, mu, ct_dt2, C_I;
    int has_s;
} or_phys;

static or_phys unpack_phys(const double phys[5])
{
    or_phys p;
    p.rho = phys[0];
    p.mu = phys[1];
    p.ct_dt2 = phys[2];
    p.C_I = phys[3];
    p.has_s = phys[4] != 0.0;
    return p;
}

/* Field values at one Gauss point of one element. */
typedef struct {
    double N[8], dN[8][3];  /* shape values, physical gradients dN_a/dx_j */
    double v[3], gv[3][3];  /* v_i, gv[i][j] = d v_i / d x_j            */
    double p, gp[3];
    double a[3], f[3], s;
    double detJ, G[3][3];   /* Jacobian determinant, metric G of Sec. 2.1 */
} gp_state;

/* Geometry at a Gauss point.  Uniform grid (Xn == NULL): dxi_k/dx_k = 2/h_k,
 * detJ = h_x h_y h_z / 8, G = diag(4/h_k^2).  Mapped grid (node coordinates
 * Xn [n][3]): J_ik = dx_i/dxi_k = sum_a x_ai dN_a/dxi_k, dN_a/dx_j =
 * sum_k dN_a/dxi_k (J^-1)_kj, G_ij = sum_k (J^-1)_ki (J^-1)_kj (Sec. 2.1).   */
static void gp_geometry(const int N[3], const double h[3], const double *Xn, int ex, int ey,
                        int ez, const double dNdxi[24], gp_state *st)
{
    if (!Xn) {
        for (int a = 0; a < 8; ++a)
            for (int j = 0; j < 3; ++j) st->dN[a][j] = dNdxi[3 * a + j] * (2.0 / h[j]);
        st->detJ = h[0] * h[1] * h[2] / 8.0;
        memset(st->G, 0, sizeof st->G);
        for (int k = 0; k < 3; ++k) st->G[k][k] = 4.0 / (h[k] * h[k]);
        return;
    }
    double J[3][3] = {{0}};
    for (int a = 0; a < 8; ++a) {
        const double *x = Xn + 3 * elem_node(N, ex, ey, ez, a);
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) J[i][k] += x[i] * dNdxi[3 * a + k];
    }
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    for (int a = 0; a < 8; ++a)
        for (int j = 0; j < 3; ++j) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += dNdxi[3 * a + k] * Ji[k][j];
            st->dN[a][j] = t;
        }
    st->detJ = det;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += Ji[k][i] * Ji[k][j];
            st->G[i][j] = t;
        }
}

static void eval_gp(const int N[3], const double h[3], const double *Xn, int ex, int ey, int ez,
                    int g, const double *U, const double *A, const double *f, int has_s,
                    gp_state *st)
{
    const double gq = 1.0 / sqrt(3.0);
    double xi[3] = {(g & 1) ? gq : -gq, (g & 2) ? gq : -gq, (g & 4) ? gq : -gq};
    double dNdxi[24];
    or_shape(xi, st->N, dNdxi);
    gp_geometry(N, h, Xn, ex, ey, ez, dNdxi, st);
    memset(st->v, 0, sizeof st->v);
    memset(st->gv, 0, sizeof st->gv);
    memset(st->gp, 0, sizeof st->gp);
    memset(st->a, 0, sizeof st->a);
    memset(st->f, 0, sizeof st->f);
    st->p = 0.0;
    st->s = has_s ? 0.0 : 1.0;
    for (int a = 0; a < 8; ++a) {
        int64_t nd = elem_node(N, ex, ey, ez, a);
        const double *u = U + 4 * nd;
        const double *ac = A + 4 * nd;
        for (int i = 0; i < 3; ++i) {
            st->v[i] += st->N[a] * u[i];
            st->a[i] += st->N[a] * ac[i];
            if (f) st->f[i] += st->N[a] * f[4 * nd + i];
            for (int j = 0; j < 3; ++j) st->gv[i][j] += st->dN[a][j] * u[i];
        }
        st->p += st->N[a] * u[3];
        for (int j = 0; j < 3; ++j) st->gp[j] += st->dN[a][j] * u[3];
        if (has_s) st->s += st->N[a] * ac[3];
    }
}

/* ------------------------------------------------------------------------ */
/* Element residual.  The weak form at a Gauss point, per test node A:
 *
 * momentum (component i):
 *     N_A rho (a_i + v_j d_j v_i - f_i)             Galerkin inertia+convection
 *   + d_j N_A mu (d_j v_i + d_i v_j)                 2 mu eps(w):eps(v)
 *   - d_i N_A p                                      -(div w, p)
 *   - rho v_j d_j N_A u'_i                           -(rho v.grad w, u')   SUPG
 *   - d_i N_A p'                                     -(div w, p')          LSIC
 *   + N_A rho u'_j d_j v_i                           (w, rho u'.grad v)    cross
 *   - rho d_j N_A u'_i u'_j                          -(grad w, rho u'(x)u') Reynolds
 * continuity:
 *     N_A d_j v_j                                    (q, div v)
 *   - d_j N_A u'_j                                   -(grad q, u')         PSPG
 *
 * with the strong residuals r_M = rho (a + v.grad v - f) + grad p,
 * r_C = div v, and the fine scales u' = -(tau_M/rho) r_M, p' = -rho tau_C r_C.
 * stab = 0 drops every term carrying u' or p' (plain Galerkin).             */
/* The weak form above at one quadrature point: st holds the shape values and
 * physical gradients of the nloc local nodes and the field values there; w is
 * the quadrature weight times det J.  Adds into Re[nloc][4].                 */
static void gp_residual(const gp_state *stp, const or_phys *ph, int nloc, double w, int stab,
                        double Re[][4])
{
    const gp_state st = *stp;
    const double rho = ph->rho, mu = ph->mu;
    double conv[3], rM[3], up[3];
    for (int i = 0; i < 3; ++i) {
        conv[i] = 0.0;
        for (int j = 0; j < 3; ++j) conv[i] += st.v[j] * st.gv[i][j];
        rM[i] = rho * (st.a[i] + conv[i] - st.f[i]) + st.gp[i];
    }
    double rC = st.gv[0][0] + st.gv[1][1] + st.gv[2][2];
    double tau[2];
    tau_of_G(st.v, st.s, st.G, rho, mu, ph->ct_dt2, ph->C_I, tau);
    double pp = 0.0;
    for (int i = 0; i < 3; ++i) up[i] = stab ? -(tau[0] / rho) * rM[i] : 0.0;
    if (stab) pp = -rho * tau[1] * rC;

    for (int A_ = 0; A_ < nloc; ++A_) {
        const double NA = st.N[A_];
        const double *dNA = st.dN[A_];
        double vgradN = 0.0;
        for (int j = 0; j < 3; ++j) vgradN += st.v[j] * dNA[j];
        for (int i = 0; i < 3; ++i) {
            double t = NA * rho * (st.a[i] + conv[i] - st.f[i]);
            for (int j = 0; j < 3; ++j) t += dNA[j] * mu * (st.gv[i][j] + st.gv[j][i]);
            t -= dNA[i] * st.p;
            t -= rho * vgradN * up[i];
            t -= dNA[i] * pp;
            for (int j = 0; j < 3; ++j) t += NA * rho * up[j] * st.gv[i][j];
            for (int j = 0; j < 3; ++j) t -= rho * dNA[j] * up[i] * up[j];
            Re[A_][i] += w * t;
        }
        double c = NA * rC;
        for (int j = 0; j < 3; ++j) c -= dNA[j] * up[j];
        Re[A_][3] += w * c;
    }
}

static void element_residual(const int N[3], const double h[3], const double *Xn,
                             const or_phys *ph, int ex, int ey, int ez, const double *U,
                             const double *A, const double *f, int stab, double Re[8][4])
{
    memset(Re, 0, 8 * 4 * sizeof(double));
    for (int g = 0; g < 8; ++g) {
        gp_state st;
        eval_gp(N, h, Xn, ex, ey, ez, g, U, A, f, ph->has_s, &st);
        gp_residual(&st, ph, 8, st.detJ, stab, Re);
    }
}

/* ------------------------------------------------------------------------ */
/* Element Jacobian-vector product: the directional derivative of the element
 * residual above in the direction dU = (c_v x_v, x_p), dA = (c_a x_v, 0),
 * i.e. the consistent linearisation with respect to (Vdot_{n+1}, P_{n+1})
 * with the generalized-alpha chain factors c_a = alpha_m and
 * c_v = alpha_f gamma dt (Sec. 2.4).  xe holds the 8x4 local direction.
 * Every term of element_residual is differentiated, including the
 * dependence of tau_M and tau_C on v.                                        */
/* The directional derivative of gp_residual at one quadrature point in the
 * direction xe[nloc][4] (velocity columns scaled by c_v in U and c_a in A,
 * pressure column unscaled); w = quadrature weight times det J.            */
static void gp_jacobian(const gp_state *stp, const or_phys *ph, int nloc, double w,
                        const double xe[][4], double c_a, double c_v, double Je[][4])
{
    const gp_state st = *stp;
    const double rho = ph->rho, mu = ph->mu;
    /* direction at the Gauss point */
    double dv[3] = {0, 0, 0}, dgv[3][3] = {{0}}, dp = 0.0, dgp[3] = {0, 0, 0};
    double da[3] = {0, 0, 0};
    for (int a = 0; a < nloc; ++a) {
        for (int i = 0; i < 3; ++i) {
            dv[i] += st.N[a] * c_v * xe[a][i];
            da[i] += st.N[a] * c_a * xe[a][i];
            for (int j = 0; j < 3; ++j) dgv[i][j] += st.dN[a][j] * c_v * xe[a][i];
        }
        dp += st.N[a] * xe[a][3];
        for (int j = 0; j < 3; ++j) dgp[j] += st.dN[a][j] * xe[a][3];
    }
    /* base state */
    double conv[3], rM[3], up[3];
    for (int i = 0; i < 3; ++i) {
        conv[i] = 0.0;
        for (int j = 0; j < 3; ++j) conv[i] += st.v[j] * st.gv[i][j];
        rM[i] = rho * (st.a[i] + conv[i] - st.f[i]) + st.gp[i];
    }
    double rC = st.gv[0][0] + st.gv[1][1] + st.gv[2][2];
    double tau[2];
    tau_of_G(st.v, st.s, st.G, rho, mu, ph->ct_dt2, ph->C_I, tau);
    double tauM = tau[0], tauC = tau[1];
    for (int i = 0; i < 3; ++i) up[i] = -(tauM / rho) * rM[i];
    /* derivatives */
    double dconv[3], drM[3], dup[3];
    for (int i = 0; i < 3; ++i) {
        dconv[i] = 0.0;
        for (int j = 0; j < 3; ++j) dconv[i] += dv[j] * st.gv[i][j] + st.v[j] * dgv[i][j];
        drM[i] = rho * (da[i] + dconv[i]) + dgp[i];
    }
    double drC = dgv[0][0] + dgv[1][1] + dgv[2][2];
    /* tau_M = (s Q)^(-1/2), Q = C_T/dt^2 + v.G v + C_I nu^2 G:G
     * d tau_M = -1/2 tau_M^3 s dQ, dQ = 2 v.G dv ;
     * tau_C = 1/(tau_M trG) -> d tau_C = -tau_C d tau_M / tau_M          */
    double dQ = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) dQ += 2.0 * st.v[i] * st.G[i][j] * dv[j];
    double dtauM = -0.5 * tauM * tauM * tauM * st.s * dQ;
    double dtauC = -tauC * dtauM / tauM;
    for (int i = 0; i < 3; ++i) dup[i] = -(dtauM * rM[i] + tauM * drM[i]) / rho;
    double dpp = -rho * (dtauC * rC + tauC * drC);

    for (int A_ = 0; A_ < nloc; ++A_) {
        const double NA = st.N[A_];
        const double *dNA = st.dN[A_];
        double vgradN = 0.0, dvgradN = 0.0;
        for (int j = 0; j < 3; ++j) {
            vgradN += st.v[j] * dNA[j];
            dvgradN += dv[j] * dNA[j];
        }
        for (int i = 0; i < 3; ++i) {
            double t = NA * rho * (da[i] + dconv[i]);
            for (int j = 0; j < 3; ++j) t += dNA[j] * mu * (dgv[i][j] + dgv[j][i]);
            t -= dNA[i] * dp;
            t -= rho * (dvgradN * up[i] + vgradN * dup[i]);
            t -= dNA[i] * dpp;
            for (int j = 0; j < 3; ++j)
                t += NA * rho * (dup[j] * st.gv[i][j] + up[j] * dgv[i][j]);
            for (int j = 0; j < 3; ++j)
                t -= rho * dNA[j] * (dup[i] * up[j] + up[i] * dup[j]);
            Je[A_][i] += w * t;
        }
        double c = NA * drC;
        for (int j = 0; j < 3; ++j) c -= dNA[j] * dup[j];
        Je[A_][3] += w * c;
    }
}

static void element_jacobian_apply(const int N[3], const double h[3], const double *Xn,
                                   const or_phys *ph, int ex, int ey, int ez, const double *U,
                                   const double *A, const double *f,
                                   const double xe[8][4], double c_a, double c_v,
                                   double Je[8][4])
{
    memset(Je, 0, 8 * 4 * sizeof(double));
    for (int g = 0; g < 8; ++g) {
        gp_state st;
        eval_gp(N, h, Xn, ex, ey, ez, g, U, A, f, ph->has_s, &st);
        gp_jacobian(&st, ph, 8, st.detJ, xe, c_a, c_v, Je);
    }
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Assembled VMS residual R[n][4] (Sec. 2.1, Eq. fluid_weak_form + VMS).
 * f may be NULL (no body force).                                            */
static void residual_drv(const int N[3], const double h[3], const double *Xn,
                         const double phys[5], const double *U, const double *A, const double *f,
                         int stab, double *R, int nthreads)
{
    or_phys ph = unpack_phys(phys);
    int64_t E = (int64_t)N[0] * N[1] * N[2];
    int64_t n = (int64_t)(N[0] + 1) * (N[1] + 1) * (N[2] + 1);
    double *Rel = (double *)malloc((size_t)E * 32 * sizeof(double));
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        int ex = (int)(e % N[0]), ey = (int)((e / N[0]) % N[1]), ez = (int)(e / ((int64_t)N[0] * N[1]));
        element_residual(N, h, Xn, &ph, ex, ey, ez, U, A, f, stab, (double(*)[4])(Rel + 32 * e));
    }
    memset(R, 0, (size_t)n * 4 * sizeof(double));
    for (int64_t e = 0; e < E; ++e) {
        int ex = (int)(e % N[0]), ey = (int)((e / N[0]) % N[1]), ez = (int)(e / ((int64_t)N[0] * N[1]));
        for (int a = 0; a < 8; ++a) {
            int64_t nd = elem_node(N, ex, ey, ez, a);
            for (int c = 0; c < 4; ++c) R[4 * nd + c] += Rel[32 * e + 4 * a + c];
        }
    }
    free(Rel);
}

/* Assembled Jacobian-vector product Jx[n][4] of or_residual (stab = 1). */
static void jacobian_drv(const int N[3], const double h[3], const double *Xn,
                         const double phys[5], const double *U, const double *A,
                         const double *f, const double *x, double c_a, double c_v, double *Jx,
                         int nthreads)
{
    or_phys ph = unpack_phys(phys);
    int64_t E = (int64_t)N[0] * N[1] * N[2];
    int64_t n = (int64_t)(N[0] + 1) * (N[1] + 1) * (N[2] + 1);
    double *Jel = (double *)malloc((size_t)E * 32 * sizeof(double));
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        int ex = (int)(e % N[0]), ey = (int)((e / N[0]) % N[1]), ez = (int)(e / ((int64_t)N[0] * N[1]));
        double xe[8][4];
        for (int a = 0; a < 8; ++a) {
            int64_t nd = elem_node(N, ex, ey, ez, a);
            for (int c = 0; c < 4; ++c) xe[a][c] = x[4 * nd + c];
        }
        element_jacobian_apply(N, h, Xn, &ph, ex, ey, ez, U, A, f, (const double(*)[4])xe, c_a,
                               c_v, (double(*)[4])(Jel + 32 * e));
    }
    memset(Jx, 0, (size_t)n * 4 * sizeof(double));
    for (int64_t e = 0; e < E; ++e) {
        int ex = (int)(e % N[0]), ey = (int)((e / N[0]) % N[1]), ez = (int)(e / ((int64_t)N[0] * N[1]));
        for (int a = 0; a < 8; ++a) {
            int64_t nd = elem_node(N, ex, ey, ez, a);
            for (int c = 0; c < 4; ++c) Jx[4 * nd + c] += Jel[32 * e + 4 * a + c];
        }
    }
    free(Jel);
}

void or_residual(const int N[3], const double h[3], const double phys[5], const double *U,
                 const double *A, const double *f, int stab, double *R, int nthreads)
{
    residual_drv(N, h, NULL, phys, U, A, f, stab, R, nthreads);
}

void or_jacobian_apply(const int N[3], const double h[3], const double phys[5],
                       const double *U, const double *A, const double *f,
                       const double *x, double c_a, double c_v, double *Jx, int nthreads)
{
    jacobian_drv(N, h, NULL, phys, U, A, f, x, c_a, c_v, Jx, nthreads);
}

/* The same operators on a mapped (curvilinear) structured grid: node
 * coordinates Xn [n][3] in the node numbering of the uniform grid, the
 * geometry of every Gauss point from the trilinear map (gp_geometry).       */
void or_residual_x(const int N[3], const double *Xn, const double phys[5], const double *U,
                   const double *A, const double *f, int stab, double *R, int nthreads)
{
    const double h[3] = {1.0, 1.0, 1.0};
    residual_drv(N, h, Xn, phys, U, A, f, stab, R, nthreads);
}

void or_jacobian_apply_x(const int N[3], const double *Xn, const double phys[5],
                         const double *U, const double *A, const double *f, const double *x,
                         double c_a, double c_v, double *Jx, int nthreads)
{
    const double h[3] = {1.0, 1.0, 1.0};
    jacobian_drv(N, h, Xn, phys, U, A, f, x, c_a, c_v, Jx, nthreads);
}

/* Element tangent matrices Ke[E][32][32], column (4b+d) = element Jacobian
 * applied to the unit direction at local node b, component d.  Used by the
 * oracle's direct Newton solves on small grids.  conn[E][8] receives the
 * global node of each local node.                                           */
static void element_jacobian_drv(const int N[3], const double h[3], const double *Xn,
                                 const double phys[5], const double *U, const double *A,
                                 const double *f, double c_a, double c_v, double *Ke,
                                 int64_t *conn, int nthreads)
{
    or_phys ph = unpack_phys(phys);
    int64_t E = (int64_t)N[0] * N[1] * N[2];
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        int ex = (int)(e % N[0]), ey = (int)((e / N[0]) % N[1]), ez = (int)(e / ((int64_t)N[0] * N[1]));
        for (int a = 0; a < 8; ++a) conn[8 * e + a] = elem_node(N, ex, ey, ez, a);
        for (int col = 0; col < 32; ++col) {
            double xe[8][4] = {{0}};
            double Je[8][4];
            xe[col / 4][col % 4] = 1.0;
            element_jacobian_apply(N, h, Xn, &ph, ex, ey, ez, U, A, f, (const double(*)[4])xe,
                                   c_a, c_v, Je);
            for (int row = 0; row < 32; ++row)
                Ke[(int64_t)1024 * e + 32 * row + col] = Je[row / 4][row % 4];
        }
    }
}

void or_element_jacobian(const int N[3], const double h[3], const double phys[5],
                         const double *U, const double *A, const double *f, double c_a,
                         double c_v, double *Ke, int64_t *conn, int nthreads)
{
    element_jacobian_drv(N, h, NULL, phys, U, A, f, c_a, c_v, Ke, conn, nthreads);
}

void or_element_jacobian_x(const int N[3], const double *Xn, const double phys[5],
                           const double *U, const double *A, const double *f, double c_a,
                           double c_v, double *Ke, int64_t *conn, int nthreads)
{
    const double h[3] = {1.0, 1.0, 1.0};
    element_jacobian_drv(N, h, Xn, phys, U, A, f, c_a, c_v, Ke, conn, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Point location on the uniform grid (the role of the point search of
 * Sec. 3 / Algorithm 1: element number and parametric position xi).
 * t_k = (X_k - x0_k)/h_k ; a point is outside unless 0 <= t_k <= N_k for all
 * k; e_k = min(floor(t_k), N_k - 1) ; xi_k = 2 (t_k - e_k) - 1.
 * Outside points get elem = -1 and xi = 0.  Returns the outside count.      */
int64_t or_locate(const int N[3], const double x0[3], const double h[3], int64_t m,
                  const double *X, int32_t *elem, double *xi)
{
    int64_t outside = 0;
    for (int64_t b = 0; b < m; ++b) {
        double t[3];
        int e[3], in = 1;
        for (int k = 0; k < 3; ++k) {
            t[k] = (X[3 * b + k] - x0[k]) / h[k];
            if (!(t[k] >= 0.0 && t[k] <= (double)N[k])) in = 0;
        }
        if (!in) {
            elem[b] = -1;
            xi[3 * b] = xi[3 * b + 1] = xi[3 * b + 2] = 0.0;
            ++outside;
            continue;
        }
        for (int k = 0; k < 3; ++k) {
            e[k] = (int)floor(t[k]);
            if (e[k] > N[k] - 1) e[k] = N[k] - 1;
            xi[3 * b + k] = 2.0 * (t[k] - (double)e[k]) - 1.0;
        }
        elem[b] = (int32_t)(e[0] + N[0] * (e[1] + N[1] * e[2]));
    }
    return outside;
}

/* Point location on a mapped structured grid (node coordinates Xn [n][3]):
 * brute force over the elements in element order; in each, Newton's method
 * on the trilinear map x(xi) = sum_a N_a(xi) x_a from xi = 0 (at most 50
 * iterations, stop when the update is below 1e-15); the point belongs to
 * the first element where the iteration settles (last update below 1e-12:
 * a root of x(xi) = X) at a xi with |xi_k| <= 1 + 1e-10.  Outside points
 * get elem = -1, xi = 0.  Returns the outside count.                        */
static int invert_trilinear(const int N[3], const double *Xn, int ex, int ey, int ez,
                            const double X[3], double xi[3])
{
    double xa[8][3];
    for (int a = 0; a < 8; ++a) {
        const double *x = Xn + 3 * elem_node(N, ex, ey, ez, a);
        for (int i = 0; i < 3; ++i) xa[a][i] = x[i];
    }
    xi[0] = xi[1] = xi[2] = 0.0;
    double last = 1.0;
    for (int it = 0; it < 50; ++it) {
        double Nv[8], dN[24], r[3] = {0, 0, 0}, J[3][3] = {{0}};
        or_shape(xi, Nv, dN);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i) {
                r[i] += Nv[a] * xa[a][i];
                for (int k = 0; k < 3; ++k) J[i][k] += xa[a][i] * dN[3 * a + k];
            }
        for (int i = 0; i < 3; ++i) r[i] -= X[i];
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(fabs(det) > 0.0)) return 0;
        double d[3];
        /* Cramer's rule for J d = r */
        d[0] = (r[0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                J[0][1] * (r[1] * J[2][2] - J[1][2] * r[2]) +
                J[0][2] * (r[1] * J[2][1] - J[1][1] * r[2])) / det;
        d[1] = (J[0][0] * (r[1] * J[2][2] - J[1][2] * r[2]) -
                r[0] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                J[0][2] * (J[1][0] * r[2] - r[1] * J[2][0])) / det;
        d[2] = (J[0][0] * (J[1][1] * r[2] - r[1] * J[2][1]) -
                J[0][1] * (J[1][0] * r[2] - r[1] * J[2][0]) +
                r[0] * (J[1][0] * J[2][1] - J[1][1] * J[2][0])) / det;
        double mx = 0.0;
        for (int k = 0; k < 3; ++k) {
            xi[k] -= d[k];
            if (fabs(d[k]) > mx) mx = fabs(d[k]);
            if (!(fabs(xi[k]) < 10.0)) return 0;
        }
        last = mx;
        if (mx < 1e-15) break;
    }
    /* a root only: an iteration that has not settled says nothing */
    if (!(last < 1e-12)) return 0;
    for (int k = 0; k < 3; ++k)
        if (!(fabs(xi[k]) <= 1.0 + 1e-10)) return 0;
    return 1;
}

int64_t or_locate_x(const int N[3], const double *Xn, int64_t m, const double *X, int32_t *elem,
                    double *xi)
{
    int64_t outside = 0;
    for (int64_t b = 0; b < m; ++b) {
        int found = 0;
        for (int ez = 0; ez < N[2] && !found; ++ez)
            for (int ey = 0; ey < N[1] && !found; ++ey)
                for (int ex = 0; ex < N[0] && !found; ++ex)
                    if (invert_trilinear(N, Xn, ex, ey, ez, X + 3 * b, xi + 3 * b)) {
                        elem[b] = ex + N[0] * (ey + N[1] * ez);
                        found = 1;
                    }
        if (!found) {
            elem[b] = -1;
            xi[3 * b] = xi[3 * b + 1] = xi[3 * b + 2] = 0.0;
            ++outside;
        }
    }
    return outside;
}

/* Cell -> points CSR by a stable counting sort on the element number:
 * cell_start[E+1], perm[m] lists the inside points cell by cell in
 * increasing point index, then the outside points in increasing index.     */
void or_cell_hash(const int N[3], int64_t m, const int32_t *elem, int32_t *cell_start,
                  int32_t *perm)
{
    int64_t E = (int64_t)N[0] * N[1] * N[2];
    memset(cell_start, 0, (size_t)(E + 1) * sizeof(int32_t));
    for (int64_t b = 0; b < m; ++b)
        if (elem[b] >= 0) cell_start[elem[b] + 1] += 1;
    for (int64_t c = 0; c < E; ++c) cell_start[c + 1] += cell_start[c];
    int32_t *cursor = (int32_t *)malloc((size_t)(E + 1) * sizeof(int32_t));
    memcpy(cursor, cell_start, (size_t)(E + 1) * sizeof(int32_t));
    int64_t tail = cell_start[E];
    for (int64_t b = 0; b < m; ++b) {
        if (elem[b] >= 0)
            perm[cursor[elem[b]]++] = (int32_t)b;
        else
            perm[tail++] = (int32_t)b;
    }
    free(cursor);
}

/* Interpolation of Eq. (nodal_solid_velo): u_B = sum_A N_A(xi_B) v_A over
 * the 8 nodes of the element holding point B (velocity components only).
 * Outside points (elem < 0) get u = 0.                                      */
void or_interp(const int N[3], int64_t m, const int32_t *elem, const double *xi,
               const double *U, double *u)
{
    for (int64_t b = 0; b < m; ++b) {
        u[3 * b] = u[3 * b + 1] = u[3 * b + 2] = 0.0;
        if (elem[b] < 0) continue;
        int e = elem[b];
        int ex = e % N[0], ey = (e / N[0]) % N[1], ez = e / (N[0] * N[1]);
        double Nv[8], dN[24];
        or_shape(xi + 3 * b, Nv, dN);
        for (int a = 0; a < 8; ++a) {
            int64_t nd = elem_node(N, ex, ey, ez, a);
            for (int i = 0; i < 3; ++i) u[3 * b + i] += Nv[a] * U[4 * nd + i];
        }
    }
}

/* Spreading with the FSI constraint matrix of Eq. (fsi_constraint_matrix):
 * F_A += sum_B w_B N_A(xi_B) lambda_B into the momentum slots; the pressure
 * slot is neither read nor written.  w may be NULL (w_B = 1).  accumulate = 0
 * first sets the momentum slots to zero.                                    */
void or_spread(const int N[3], int64_t m, const int32_t *elem, const double *xi,
               const double *lam, const double *w, double *F, int accumulate)
{
    int64_t n = (int64_t)(N[0] + 1) * (N[1] + 1) * (N[2] + 1);
    if (!accumulate)
        for (int64_t a = 0; a < n; ++a) F[4 * a] = F[4 * a + 1] = F[4 * a + 2] = 0.0;
    for (int64_t b = 0; b < m; ++b) {
        if (elem[b] < 0) continue;
        int e = elem[b];
        int ex = e % N[0], ey = (e / N[0]) % N[1], ez = e / (N[0] * N[1]);
        double Nv[8], dN[24];
        or_shape(xi + 3 * b, Nv, dN);
        double wb = w ? w[b] : 1.0;
        for (int a = 0; a < 8; ++a) {
            int64_t nd = elem_node(N, ex, ey, ez, a);
            for (int i = 0; i < 3; ++i) F[4 * nd + i] += wb * Nv[a] * lam[3 * b + i];
        }
    }
}

/* ======================================================================== */
/* Unstructured tetrahedral background meshes: linear (P1-P1) tetrahedra,    */
/* the element family of the paper's valve fluid mesh (Sec. 4).              */
/*                                                                          */
/* Nodes X[n][3], elements tets[E][4] (node numbers, any orientation).       */
/* Reference tetrahedron with vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1):   */
/* N_0 = 1 - xi_1 - xi_2 - xi_3, N_k = xi_k.  J_ik = dx_i/dxi_k =            */
/* x_{k,i} - x_{0,i}; dN_a/dx_j = sum_k dN_a/dxi_k (J^-1)_kj; the metric of   */
/* Sec. 2.1 is G = J^-T J^-1 with the reference tetrahedron as the parent    */
/* domain.  Quadrature: the symmetric 4-point rule of degree 2, barycentric  */
/* coordinates (al, be, be, be) and permutations, al = (5 + 3 sqrt 5)/20,    */
/* be = (5 - sqrt 5)/20, each with weight |det J|/24 (the volume / 4).      */
/* The weak form per quadrature point is gp_residual / gp_jacobian, the same */
/* as on hexahedra.  On P1 elements the gradients are constant per element,  */
/* so the dropped viscous term of r_M is exactly zero here.                  */
/* ======================================================================== */

static void tet_geometry(const double *X, const int32_t *t, double dN[4][3], double *det,
                         double G[3][3])
{
    double J[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) J[i][k] = X[3 * t[k + 1] + i] - X[3 * t[0] + i];
    double d = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
    /* dN_k/dx_j = (J^-1)_{k-1,j} for k = 1..3, dN_0 = -(sum of the others) */
    for (int j = 0; j < 3; ++j) {
        dN[1][j] = Ji[0][j];
        dN[2][j] = Ji[1][j];
        dN[3][j] = Ji[2][j];
        dN[0][j] = -(Ji[0][j] + Ji[1][j] + Ji[2][j]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ji[k][i] * Ji[k][j];
            G[i][j] = s;
        }
    *det = d;
}

static void eval_qp_tet(const double *X, const int32_t *t, int q, const double *U,
                        const double *A, const double *f, int has_s, gp_state *st)
{
    const double al = (5.0 + 3.0 * sqrt(5.0)) / 20.0, be = (5.0 - sqrt(5.0)) / 20.0;
    memset(st, 0, sizeof *st);
    double det;
    tet_geometry(X, t, st->dN, &det, st->G);
    st->detJ = det;
    st->s = has_s ? 0.0 : 1.0;
    for (int a = 0; a < 4; ++a) {
        st->N[a] = (a == q) ? al : be;
        const int64_t nd = t[a];
        const double *u = U + 4 * nd;
        const double *ac = A + 4 * nd;
        for (int i = 0; i < 3; ++i) {
            st->v[i] += st->N[a] * u[i];
            st->a[i] += st->N[a] * ac[i];
            if (f) st->f[i] += st->N[a] * f[4 * nd + i];
            for (int j = 0; j < 3; ++j) st->gv[i][j] += st->dN[a][j] * u[i];
        }
        st->p += st->N[a] * u[3];
        for (int j = 0; j < 3; ++j) st->gp[j] += st->dN[a][j] * u[3];
        if (has_s) st->s += st->N[a] * ac[3];
    }
}

static void tet_element_residual(const double *X, const int32_t *t, const or_phys *ph,
                                 const double *U, const double *A, const double *f, int stab,
                                 double Re[4][4])
{
    memset(Re, 0, 16 * sizeof(double));
    for (int q = 0; q < 4; ++q) {
        gp_state st;
        eval_qp_tet(X, t, q, U, A, f, ph->has_s, &st);
        gp_residual(&st, ph, 4, fabs(st.detJ) / 24.0, stab, Re);
    }
}

static void tet_element_jacobian_apply(const double *X, const int32_t *t, const or_phys *ph,
                                       const double *U, const double *A, const double *f,
                                       const double xe[4][4], double c_a, double c_v,
                                       double Je[4][4])
{
    memset(Je, 0, 16 * sizeof(double));
    for (int q = 0; q < 4; ++q) {
        gp_state st;
        eval_qp_tet(X, t, q, U, A, f, ph->has_s, &st);
        gp_jacobian(&st, ph, 4, fabs(st.detJ) / 24.0, xe, c_a, c_v, Je);
    }
}

/* Assembled residual R[n][4] on a tetrahedral mesh (element contributions in
 * parallel, assembly serial in element order).                              */
void or_tet_residual(int64_t n, const double *X, int64_t E, const int32_t *tets,
                     const double phys[5], const double *U, const double *A, const double *f,
                     int stab, double *R, int nthreads)
{
    or_phys ph = unpack_phys(phys);
    double *Rel = (double *)malloc((size_t)E * 16 * sizeof(double));
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e)
        tet_element_residual(X, tets + 4 * e, &ph, U, A, f, stab, (double(*)[4])(Rel + 16 * e));
    memset(R, 0, (size_t)n * 4 * sizeof(double));
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 4; ++c) R[4 * (int64_t)tets[4 * e + a] + c] += Rel[16 * e + 4 * a + c];
    free(Rel);
}

/* Assembled Jacobian-vector product Jx[n][4] (stab = 1), chain factors c_a,
 * c_v as on hexahedra.                                                        */
void or_tet_jacobian_apply(int64_t n, const double *X, int64_t E, const int32_t *tets,
                           const double phys[5], const double *U, const double *A,
                           const double *f, const double *x, double c_a, double c_v, double *Jx,
                           int nthreads)
{
    or_phys ph = unpack_phys(phys);
    double *Jel = (double *)malloc((size_t)E * 16 * sizeof(double));
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        const int32_t *t = tets + 4 * e;
        double xe[4][4];
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 4; ++c) xe[a][c] = x[4 * (int64_t)t[a] + c];
        tet_element_jacobian_apply(X, t, &ph, U, A, f, (const double(*)[4])xe, c_a, c_v,
                                   (double(*)[4])(Jel + 16 * e));
    }
    memset(Jx, 0, (size_t)n * 4 * sizeof(double));
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 4; ++c)
                Jx[4 * (int64_t)tets[4 * e + a] + c] += Jel[16 * e + 4 * a + c];
    free(Jel);
}

/* Element Jacobians Ke[E][16][16] (row = 4 a + c of the residual, column =
 * 4 b + d of the direction), by applying the element linearisation to the
 * 16 unit directions.                                                        */
void or_tet_element_jacobian(const double *X, int64_t E, const int32_t *tets,
                             const double phys[5], const double *U, const double *A,
                             const double *f, double c_a, double c_v, double *Ke, int nthreads)
{
    or_phys ph = unpack_phys(phys);
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e)
        for (int col = 0; col < 16; ++col) {
            double xe[4][4] = {{0}};
            double Je[4][4];
            xe[col / 4][col % 4] = 1.0;
            tet_element_jacobian_apply(X, tets + 4 * e, &ph, U, A, f, (const double(*)[4])xe,
                                       c_a, c_v, Je);
            for (int row = 0; row < 16; ++row)
                Ke[(int64_t)256 * e + 16 * row + col] = Je[row / 4][row % 4];
        }
}

/* Barycentric coordinates of P in tetrahedron t: with e_k = x_k - x_0 and
 * d = P - x_0, lam_1 = d.(e2 x e3)/D, lam_2 = e1.(d x e3)/D,
 * lam_3 = e1.(e2 x d)/D, D = e1.(e2 x e3), lam_0 = 1 - lam_1 - lam_2 - lam_3,
 * each product and sum evaluated left to right as written.                   */
void or_tet_barycentric(const double *X, const int32_t *t, const double P[3], double lam[4])
{
    double e1[3], e2[3], e3[3], d[3];
    for (int i = 0; i < 3; ++i) {
        e1[i] = X[3 * t[1] + i] - X[3 * t[0] + i];
        e2[i] = X[3 * t[2] + i] - X[3 * t[0] + i];
        e3[i] = X[3 * t[3] + i] - X[3 * t[0] + i];
        d[i] = P[i] - X[3 * t[0] + i];
    }
    /* c = e2 x e3 */
    double c0 = e2[1] * e3[2] - e2[2] * e3[1];
    double c1 = e2[2] * e3[0] - e2[0] * e3[2];
    double c2 = e2[0] * e3[1] - e2[1] * e3[0];
    double D = e1[0] * c0 + e1[1] * c1 + e1[2] * c2;
    double l1 = (d[0] * c0 + d[1] * c1 + d[2] * c2) / D;
    /* d x e3 and e2 x d */
    double a0 = d[1] * e3[2] - d[2] * e3[1];
    double a1 = d[2] * e3[0] - d[0] * e3[2];
    double a2 = d[0] * e3[1] - d[1] * e3[0];
    double l2 = (e1[0] * a0 + e1[1] * a1 + e1[2] * a2) / D;
    double b0 = e2[1] * d[2] - e2[2] * d[1];
    double b1 = e2[2] * d[0] - e2[0] * d[2];
    double b2 = e2[0] * d[1] - e2[1] * d[0];
    double l3 = (e1[0] * b0 + e1[1] * b1 + e1[2] * b2) / D;
    lam[1] = l1;
    lam[2] = l2;
    lam[3] = l3;
    lam[0] = 1.0 - l1 - l2 - l3;
}

/* Point location on a tetrahedral mesh (the point search of Sec. 3 /
 * Algorithm 1): brute force over the elements in element order; the point
 * belongs to the first tetrahedron whose four barycentric coordinates are all
 * >= -1e-12.  lam_out[m][3] = (lam_1, lam_2, lam_3) of that element.
 * Outside points get elem = -1 and zeros.  Returns the outside count.        */
int64_t or_tet_locate(const double *X, int64_t E, const int32_t *tets, int64_t m,
                      const double *P, int32_t *elem, double *lam_out)
{
    int64_t outside = 0;
    for (int64_t b = 0; b < m; ++b) {
        int found = 0;
        for (int64_t e = 0; e < E && !found; ++e) {
            double lam[4];
            or_tet_barycentric(X, tets + 4 * e, P + 3 * b, lam);
            if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
                elem[b] = (int32_t)e;
                lam_out[3 * b] = lam[1];
                lam_out[3 * b + 1] = lam[2];
                lam_out[3 * b + 2] = lam[3];
                found = 1;
            }
        }
        if (!found) {
            elem[b] = -1;
            lam_out[3 * b] = lam_out[3 * b + 1] = lam_out[3 * b + 2] = 0.0;
            ++outside;
        }
    }
    return outside;
}

/* Interpolation u_B = sum_a N_a(lam_B) v_a (Eq. nodal_solid_velo) on
 * tetrahedra, N_0 = 1 - lam_1 - lam_2 - lam_3, N_k = lam_k.                  */
void or_tet_interp(const int32_t *tets, int64_t m, const int32_t *elem, const double *lam,
                   const double *U, double *u)
{
    for (int64_t b = 0; b < m; ++b) {
        u[3 * b] = u[3 * b + 1] = u[3 * b + 2] = 0.0;
        if (elem[b] < 0) continue;
        const int32_t *t = tets + 4 * (int64_t)elem[b];
        const double l1 = lam[3 * b], l2 = lam[3 * b + 1], l3 = lam[3 * b + 2];
        const double Nv[4] = {1.0 - l1 - l2 - l3, l1, l2, l3};
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) u[3 * b + i] += Nv[a] * U[4 * (int64_t)t[a] + i];
    }
}

/* Spreading F_a += w_B N_a(lam_B) lambda_B (Eq. fsi_constraint_matrix) on
 * tetrahedra, velocity slots only; accumulate = 0 zeroes them first.        */
void or_tet_spread(int64_t n, const int32_t *tets, int64_t m, const int32_t *elem,
                   const double *lam, const double *lamv, const double *w, double *F,
                   int accumulate)
{
    if (!accumulate)
        for (int64_t a = 0; a < n; ++a) F[4 * a] = F[4 * a + 1] = F[4 * a + 2] = 0.0;
    for (int64_t b = 0; b < m; ++b) {
        if (elem[b] < 0) continue;
        const int32_t *t = tets + 4 * (int64_t)elem[b];
        const double l1 = lam[3 * b], l2 = lam[3 * b + 1], l3 = lam[3 * b + 2];
        const double Nv[4] = {1.0 - l1 - l2 - l3, l1, l2, l3};
        const double wb = w ? w[b] : 1.0;
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) F[4 * (int64_t)t[a] + i] += wb * Nv[a] * lamv[3 * b + i];
    }
}
