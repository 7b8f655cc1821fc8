"""The oracle's pins are sensitive: each plausible mistake, planted in a copy of the
oracle's C source on the CPU, makes at least one of the oracle pin tests fail.

Every mutant below changes one term of the scheme (a sign, an index order, a
dropped term, a wrong bed level, a wrong factor).  The copy is compiled into a
temporary directory and the pin suite is run against it in a subprocess.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "zoomy_oracle.c")

MUTANTS = {
    "nc_sign": ("double ea = (k == l) ? -al[0] : 0.0;", "double ea = (k == l) ? al[0] : 0.0;"),
    "nc_index_order": ("ea += al[j] * md->B[(k * m + j) * m + l] / md->M[k];",
                       "ea += al[j] * md->B[(k * m + l) * m + j] / md->M[k];"),
    "nc_y_dropped": ("Bn[ib(md, k) * nv + ib(md, l)] += ny * eb;", "(void)eb;"),
    "pressure_correction_dropped": ("out[ia(md, 0)] -= p * nx;", "(void)p;"),
    "bed_min_instead_of_max": ("double bf = bi > bj ? bi : bj;", "double bf = bi < bj ? bi : bj;"),
    "dissipation_dropped": ("out[v] = 0.5 * (Fi[v] + Fj[v]) - 0.5 * sf * dq[v];", "out[v] = 0.5 * (Fi[v] + Fj[v]);"),
    "newtonian_sign": ("S[ia(md, k)] = -(md->nu / (md->rho * h)) * sa / md->M[k];",
                       "S[ia(md, k)] = (md->nu / (md->rho * h)) * sa / md->M[k];"),
    "slip_weight_without_2k1": ("double w = md->phi0[k] / md->M[k];", "double w = md->phi0[k];"),
    "wavespeed_drops_higher_moments": ("if (k >= 2) s1 += sqrt(ak2);", "(void)s1;"),
    "wall_not_reflecting": ("if (bc != 1) return;", "return;"),
    "flux_moment_mass_matrix": ("F[ia(md, k)] = nx * (h * saa / md->M[k] + p);", "F[ia(md, k)] = nx * (h * saa + p);"),
    "rk2_average_dropped": ("for (int64_t k = 0; k < n; ++k) Q[k] = 0.5 * (Q[k] + Q2[k]);",
                           "for (int64_t k = 0; k < n; ++k) Q[k] = Q2[k];"),
    "hr_depth_not_clipped": ("if (hs < 0.0) hs = 0.0;", "(void)0;"),
    "tri_normal_y_flipped": ("me->fny[t * 3 + f] = -ex / len;", "me->fny[t * 3 + f] = ex / len;"),
    "tri_edge_length_unit": ("me->flen[t * 3 + f] = len;", "me->flen[t * 3 + f] = 1.0;"),
    "tri_area_doubled": ("me->area[t] = sa;", "me->area[t] = 2.0 * sa;"),
    "lift_w_sign": ("double w = -G + u * (gx[nv]", "double w = G + u * (gx[nv]"),
    "lift_depth_gradient_unscaled": ("u * (gx[nv] + zeta[jz] * gx[0])", "u * (gx[nv] + gx[0])"),
    "lift_phi_for_Phi": ("G += gx[ia(md, k)] * Phi[k];", "G += gx[ia(md, k)] * phi[k];"),
    "implicit_friction_sign": ("A[k][i] = (k == i ? 1.0 : 0.0) +", "A[k][i] = (k == i ? 1.0 : 0.0) -"),
    "implicit_newtonian_without_mass_matrix": ("nuh * md->Cm[i * m + k] / md->M[k]", "nuh * md->Cm[i * m + k]"),
    "order2_interior_pressure_dropped": ("acc[row] += len * 0.5 * md->g * (qp[0] + qm[0]) * (etap - etam);",
                                         "(void)row;"),
    "order2_interior_nc_dropped": ("            acc[r] += len * a;", "            (void)a;"),
    "order2_slopes_unlimited": ("minmod(wi[v] - wl[v], wr[v] - wi[v])", "0.5 * (wr[v] - wl[v])"),
    "order2_face_bed_not_reconstructed": ("*bf = bi + 0.5 * s * (sig[1] - sig[0]);", "*bf = bi;"),
    "closure_schedule_ignored_in_stage2": ("closure_stage(m4, cl, me, A, bed, dt, P, B);",
                                           "closure_stage(m4, cl, me, A, bed, dt, NULL, B);"),
    "closure_schedule1_drops_alpha2": ("closure_close(m4, q1, pred + 6 * i, q4, ah, bh);",
                                            "closure_close(m4, q1, pred + 6 * i, q4, ah, bh), q4[ia(m4, 2)] = 0.0;"),
}

FIRST_PIN = {"tri_": "tests/test_oracle_triangles.py", "lift_": "tests/test_oracle_lift.py",
             "closure_": "tests/test_oracle_closure.py",
             "implicit_": "tests/test_oracle_source.py", "order2_": "tests/test_oracle_order2.py"}
PIN_TESTS = ["tests/test_oracle_basis.py", "tests/test_oracle_model.py", "tests/test_oracle_scheme.py",
             "tests/test_oracle_triangles.py", "tests/test_oracle_lift.py", "tests/test_oracle_source.py",
             "tests/test_oracle_order2.py"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", str(mutated),
                    "-o", str(so), "-lm"], check=True, capture_output=True)
    env = dict(os.environ, ZOOMY_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    # the pin file of the mutated part first (one failing pin is enough); all pins otherwise
    first = [FIRST_PIN[p] for p in FIRST_PIN if name.startswith(p)]
    for files in ([first[0]] if first else []) + [PIN_TESTS]:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *files],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
        if r.returncode != 0:
            return
    assert False, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
