"""Independent evaluation of the VMS weak form used to pin the oracle.

This is written from the inner-product statement of the residual-based VMS
form (Bazilevs et al. 2007, the form Sec. 2.1 of the paper refers to), not
from the oracle's expanded per-node coefficients:

  B(w,q; v,p) = (w, rho a) + (w, rho v.grad v) + (eps(w), 2 mu eps(v)) - (div w, p)
              + (q, div v) - (rho v.grad w + grad q, u') - (div w, p')
              + (w, rho u'.grad v) - (grad w, rho u' (x) u') - (w, rho f)

with u' = -(tau_M/rho) r_M and p' = -rho tau_C r_C.  Integration uses a
4x4x4 Gauss-Legendre rule (different points from the 2x2x2 rule of the
method) and its own tensor-product shape functions; on fields where every
integrand is a polynomial of degree <= 3 per direction both rules are exact,
so the two evaluations agree to rounding.
"""
import numpy as np


def lagrange_1d(xi):
    """Values and derivatives of the two 1D linear Lagrange functions."""
    l = np.stack([(1 - xi) / 2, (1 + xi) / 2])
    d = np.stack([-0.5 * np.ones_like(xi), 0.5 * np.ones_like(xi)])
    return l, d


def q1_basis(pts):
    """N[q,8], dN/dxi[q,8,3] at parent points pts[q,3]."""
    lx, dx = lagrange_1d(pts[:, 0])
    ly, dy = lagrange_1d(pts[:, 1])
    lz, dz = lagrange_1d(pts[:, 2])
    N = np.empty((len(pts), 8))
    dN = np.empty((len(pts), 8, 3))
    for a in range(8):
        i, j, k = a & 1, (a >> 1) & 1, (a >> 2) & 1
        N[:, a] = lx[i] * ly[j] * lz[k]
        dN[:, a, 0] = dx[i] * ly[j] * lz[k]
        dN[:, a, 1] = lx[i] * dy[j] * lz[k]
        dN[:, a, 2] = lx[i] * ly[j] * dz[k]
    return N, dN


def gauss_rule(order):
    x, w = np.polynomial.legendre.leggauss(order)
    P = np.array([(a, b, c) for c in x for b in x for a in x])
    W = np.array([wa * wb * wc for wc in w for wb in w for wa in w])
    return P, W


def element_weak_form(h, Ue, Ae, fe, rho, mu, tau_m, tau_c, stab=True, order=4):
    """Element residual [8,4] of B above for one element of size h[3].

    Ue, Ae, fe: [8,4] nodal values (v|p, a|s, f|-) in local node order
    a = ax + 2 ay + 4 az.  tau_m, tau_c: callables of the quadrature data
    returning arrays [q] (the caller guarantees they are what the method
    evaluates).
    """
    P, W = gauss_rule(order)
    N, dNxi = q1_basis(P)
    h = np.asarray(h, dtype=float)
    dN = dNxi * (2.0 / h)[None, None, :]
    detJ = np.prod(h) / 8.0
    v = N @ Ue[:, :3]                       # [q,3]
    gv = np.einsum("qaj,ai->qij", dN, Ue[:, :3])   # gv[q,i,j] = d_j v_i
    p = N @ Ue[:, 3]
    gp = np.einsum("qaj,a->qj", dN, Ue[:, 3])
    acc = N @ Ae[:, :3]
    f = N @ fe[:, :3]
    eps_v = 0.5 * (gv + np.swapaxes(gv, 1, 2))
    div_v = np.trace(gv, axis1=1, axis2=2)
    conv = np.einsum("qj,qij->qi", v, gv)
    r_M = rho * (acc + conv - f) + gp
    r_C = div_v
    tm = tau_m(v) if stab else np.zeros(len(P))
    tc = tau_c(v) if stab else np.zeros(len(P))
    up = -(tm / rho)[:, None] * r_M
    pp = -rho * tc * r_C
    R = np.zeros((8, 4))
    for A in range(8):
        for i in range(3):
            w = np.zeros((len(P), 3))
            w[:, i] = N[:, A]
            gw = np.zeros((len(P), 3, 3))
            gw[:, i, :] = dN[:, A, :]       # (grad w)_{kl} = d_l w_k
            eps_w = 0.5 * (gw + np.swapaxes(gw, 1, 2))
            div_w = np.trace(gw, axis1=1, axis2=2)
            v_grad_w = np.einsum("qj,qkj->qk", v, gw)
            integrand = (
                np.einsum("qk,qk->q", w, rho * (acc + conv - f))
                + 2.0 * mu * np.einsum("qkl,qkl->q", eps_w, eps_v)
                - div_w * p
                - np.einsum("qk,qk->q", rho * v_grad_w, up)
                - div_w * pp
                + np.einsum("qk,qk->q", w, rho * np.einsum("qj,qkj->qk", up, gv))
                - np.einsum("qkl,qk,ql->q", gw, rho * up, up)
            )
            R[A, i] = detJ * np.sum(W * integrand)
        q_val = N[:, A]
        gq = dN[:, A, :]
        integrand = q_val * div_v - np.einsum("qj,qj->q", gq, up)
        R[A, 3] = detJ * np.sum(W * integrand)
    return R
