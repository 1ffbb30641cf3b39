"""Plant plausible mistakes in a copy of the Python oracle modules (the
immersed solid, the Schur preconditioner's pressure multigrid, the
tetrahedral pressure operator and the interface band) and check that their pins catch each one.  The oracle package
and the pin files are copied to a temporary directory and patched there; the
committed oracle is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name -> (module, anchor, replacement, pin file)
MUTATIONS = {
    "solid_P_transposed": ("solid.py", "+ lam * math.log(J) * Finv_T\n",
                           "+ lam * math.log(J) * Finv_T.T\n", "test_oracle_solid.py"),
    "solid_force_transposed": ("solid.py", "f[mesh.conn[e]] += det0 * gX @ P.T",
                               "f[mesh.conn[e]] += det0 * gX @ P", "test_oracle_solid.py"),
    "solid_tangent_term_dropped": ("solid.py", "+ lam * np.trace(Finv @ dF) * Finv_T)",
                                   ")", "test_oracle_solid.py"),
    "solid_viscous_unsymmetrised": ("solid.py", "D = 0.5 * (L + L.T)", "D = L",
                                    "test_oracle_solid.py"),
    "solid_gravity_sign": ("solid.py", "np.outer(N, ag - f)", "np.outer(N, ag + f)",
                           "test_oracle_solid.py"),
    "solid_newmark_beta": ("solid.py", "beta = 0.25 * (1.0 + am - af) ** 2",
                           "beta = 0.25 * (1.0 + am + af) ** 2", "test_oracle_solid.py"),
    "precond_prolongation_weights": ("precond.py", "[(i // 2, 0.5), (i // 2 + 1, 0.5)]",
                                     "[(i // 2, 0.25), (i // 2 + 1, 0.75)]",
                                     "test_oracle_precond.py"),
    "precond_mass_without_det": ("precond.py", "Me += detJ * np.outer(N, N)",
                                 "Me += np.outer(N, N)", "test_oracle_precond.py"),
    "precond_chebyshev_recurrence": ("precond.py", "rho_new = 1.0 / (2.0 * s1 - rho)",
                                     "rho_new = 1.0 / (2.0 * s1 + rho)", "test_oracle_precond.py"),
    "precond_sigma_chain": ("precond.py", "return af * gm * dt / (am * rho)",
                            "return gm * dt / (am * rho)", "test_oracle_precond.py"),
    "tet_pressure_mass_diagonal": ("tet.py", "(np.ones((4, 4)) + np.eye(4))[None] / 20.0",
                                   "np.ones((4, 4))[None] / 20.0", "test_oracle_tet_pressure.py"),
    "tet_pressure_gradient_index": ("tet.py", "grad = np.transpose(C[:, 1:, :], (0, 2, 1))",
                                    "grad = C[:, :, 1:]", "test_oracle_tet_pressure.py"),
    "tet_pressure_volume_factor": ("tet.py", "V = np.abs(np.linalg.det(M4)) / 6.0",
                                   "V = np.abs(np.linalg.det(M4)) / 2.0",
                                   "test_oracle_tet_pressure.py"),
    "tet_pressure_elimination_rows_only": (
        "tet.py", "keep = (A.row == A.col) | ~(el[A.row] | el[A.col])",
        "keep = (A.row == A.col) | ~el[A.row]", "test_oracle_tet_pressure.py"),
    "mapped_pressure_jacobian_transposed": (
        "precond.py", 'G = np.einsum("ad,edi->eai", dN, Jinv)',
        'G = np.einsum("ad,eid->eai", dN, Jinv)', "test_oracle_mapped_pressure.py"),
    "mapped_pressure_no_det": (
        "precond.py", "w = np.abs(np.linalg.det(J))[:, None, None]",
        "w = np.ones((J.shape[0], 1, 1))", "test_oracle_mapped_pressure.py"),
    "mapped_pressure_mass_diagonal": (
        "precond.py", "kappa * np.outer(Nq, Nq)[None])",
        "kappa * np.diag(Nq * Nq)[None])", "test_oracle_mapped_pressure.py"),
    "band_dilation_short": ("interface.py", "max(0, i - layers):min(Nx, i + layers + 1)",
                            "max(0, i - layers):min(Nx, i + layers)", "test_oracle_interface.py"),
    "band_lower_corner_only": ("interface.py", "on[dk:dk + Nz, dj:dj + Ny, di:di + Nx] |= band",
                               "on[0:Nz, 0:Ny, 0:Nx] |= band", "test_oracle_interface.py"),
}


@pytest.fixture(scope="module")
def oracle_lib():
    sys.path.insert(0, ROOT)
    import oracle.core
    return oracle.core.build()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path, oracle_lib):
    module, old, new, pin = MUTATIONS[name]
    stage_copy(tmp_path)
    src = (tmp_path / "oracle" / module).read_text()
    assert old in src, f"mutation anchor for {name} no longer in oracle/{module}"
    (tmp_path / "oracle" / module).write_text(src.replace(old, new, 1))
    r = run_pins(tmp_path, pin, oracle_lib)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
    assert r.returncode != 0, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"


def stage_copy(tmp_path):
    """The oracle package, the seeded input generators and the pin files in a
    scratch directory of their own."""
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so"))
    (tmp_path / "paper_2601_08266_gb300").mkdir()
    (tmp_path / "paper_2601_08266_gb300" / "__init__.py").write_text("")
    shutil.copy(os.path.join(ROOT, "paper_2601_08266_gb300", "inputs.py"),
                tmp_path / "paper_2601_08266_gb300" / "inputs.py")
    (tmp_path / "tests").mkdir()
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f in ("conftest.py", "weakform_ref.py") or f.startswith("test_oracle_"):
            shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)


def run_pins(tmp_path, pin, oracle_lib):
    env = dict(os.environ, FSI_ORACLE_LIB=oracle_lib)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           "-m", "not slow", f"tests/{pin}"],
                          cwd=tmp_path, env=env, capture_output=True, text=True, timeout=900)


@pytest.mark.parametrize("pin", sorted({m[3] for m in MUTATIONS.values()}))
def test_unpatched_copy_passes_its_pins(pin, tmp_path, oracle_lib):
    """Control: the staged copy without a mistake passes, so the failures above
    come from the planted mistakes."""
    stage_copy(tmp_path)
    r = run_pins(tmp_path, pin, oracle_lib)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
