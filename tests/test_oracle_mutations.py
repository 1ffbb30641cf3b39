"""Plant plausible mistakes in a copy of the C oracle and check that the pins
catch each one (a sign flip, a transposed gradient, a dropped term, a wrong
index, a dropped tau derivative).  The mistakes are planted on the CPU in a
temporary copy; the committed oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "cross_term_sign": ("t += NA * rho * up[j] * st.gv[i][j];",
                        "t -= NA * rho * up[j] * st.gv[i][j];"),
    "convection_transposed": ("conv[i] += st.v[j] * st.gv[i][j];\n        rM[i]",
                              "conv[i] += st.v[j] * st.gv[j][i];\n        rM[i]"),
    "supg_sign": ("t -= rho * vgradN * up[i];", "t += rho * vgradN * up[i];"),
    "lsic_dropped": ("t -= dNA[i] * pp;", ";"),
    "reynolds_index": ("t -= rho * dNA[j] * up[i] * up[j];",
                       "t -= rho * dNA[i] * up[j] * up[j];"),
    "pspg_sign": ("for (int j = 0; j < 3; ++j) c -= dNA[j] * up[j];\n        Re",
                  "for (int j = 0; j < 3; ++j) c += dNA[j] * up[j];\n        Re"),
    "viscous_not_symmetric": ("t += dNA[j] * mu * (st.gv[i][j] + st.gv[j][i]);",
                              "t += dNA[j] * mu * (st.gv[i][j] + st.gv[i][j]);"),
    "tau_time_term_dropped": ("sqrt(s * (ct_dt2 + vGv", "sqrt(s * (0.0 * ct_dt2 + vGv"),
    "jacobian_dtau_dropped": ("double dtauM = -0.5 * tauM * tauM * tauM * st.s * dQ;",
                              "double dtauM = 0.0;"),
    "interp_node_order": ("return node_id(N, ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1));",
                          "return node_id(N, ex + ((a >> 1) & 1), ey + (a & 1), ez + ((a >> 2) & 1));"),
    "locate_xi_sign": ("xi[3 * b + k] = 2.0 * (t[k] - (double)e[k]) - 1.0;",
                       "xi[3 * b + k] = 1.0 - 2.0 * (t[k] - (double)e[k]);"),
    # mapped grids: caught by the pins of tests/test_oracle_mapped.py
    "mapped_gradient_transposed": ("t += dNdxi[3 * a + k] * Ji[k][j];",
                                   "t += dNdxi[3 * a + k] * Ji[j][k];"),
    "mapped_metric_transposed": ("t += Ji[k][i] * Ji[k][j];", "t += Ji[i][k] * Ji[j][k];"),
    "mapped_det_dropped": ("st->detJ = det;", "st->detJ = 1.0;"),
    "mapped_locate_unsettled": ("if (!(last < 1e-12)) return 0;", ";"),
    # tetrahedra: caught by the pins of tests/test_oracle_tet.py
    "tet_quadrature_weight": ("gp_residual(&st, ph, 4, fabs(st.detJ) / 24.0, stab, Re);",
                              "gp_residual(&st, ph, 4, fabs(st.detJ) / 6.0, stab, Re);"),
    "tet_gradient_node0": ("dN[0][j] = -(Ji[0][j] + Ji[1][j] + Ji[2][j]);",
                           "dN[0][j] = (Ji[0][j] + Ji[1][j] + Ji[2][j]);"),
    "tet_quadrature_points_swapped": ("st->N[a] = (a == q) ? al : be;",
                                      "st->N[a] = (a == q) ? be : al;"),
    "tet_metric_transposed": ("s += Ji[k][i] * Ji[k][j];", "s += Ji[i][k] * Ji[j][k];"),
    "tet_jacobian_weight": ("gp_jacobian(&st, ph, 4, fabs(st.detJ) / 24.0, xe, c_a, c_v, Je);",
                            "gp_jacobian(&st, ph, 4, st.detJ / 24.0, xe, c_a, c_v, Je);"),
    "tet_locate_lam0_ignored": ("if (lam[0] >= -1e-12 && lam[1] >= -1e-12",
                                "if (1 && lam[1] >= -1e-12"),
}
MAPPED = {k for k in MUTATIONS if k.startswith("mapped_")}
TET = {k for k in MUTATIONS if k.startswith("tet_")}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "fsi_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert old in src, f"mutation anchor for {name} no longer in the oracle"
    (tmp_path / "fsi_oracle.c").write_text(src.replace(old, new, 1))
    lib = tmp_path / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                           str(tmp_path / "fsi_oracle.c"), "-lm"])
    env = dict(os.environ, FSI_ORACLE_LIB=str(lib))
    files = (["tests/test_oracle_mapped.py"] if name in MAPPED
             else ["tests/test_oracle_tet.py"] if name in TET
             else ["tests/test_oracle_vms.py", "tests/test_oracle_dlm.py"])
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        *files, "-k", "not manufactured and not quadratic"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"
