"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, index or operand, a transposed tensor), compiles the copy,
and runs, against it, the pin that should catch it (one test of
``tests/test_oracle_*.py``, in a subprocess that loads the copy through
``BD_ORACLE_LIB``). The case passes when that pin fails. The committed oracle
is untouched: the mistakes exist only in temporary copies.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (name, original source text, planted text, pin that must fail)
PLANTED = [
    # Philox4x32-10 (Salmon et al., SC'11, Sec. 4)
    ("philox_wrong_word", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c3 ^ k0;",
     "test_oracle_noise.py::test_philox_matches_curand_over_two_counter_rounds[0]"),
    ("philox_key_bump", "k1 += W1;", "k1 += W0;",
     "test_oracle_noise.py::test_philox_matches_curand_over_two_counter_rounds[0]"),
    # counter word 3 (the chain id) entering the rounds wrongly: invisible to
    # the cuRAND layout, whose word 3 is always 0
    ("philox_word3_into_word1", "uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];",
     "uint32_t c0 = ctr[0], c1 = ctr[1] ^ ctr[3], c2 = ctr[2], c3 = 0;",
     "test_oracle_noise.py::test_philox_matches_triton_on_all_four_counter_words"),
    ("philox_word3_scaled", "uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];",
     "uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3] * 3u;",
     "test_oracle_noise.py::test_philox_matches_triton_on_all_four_counter_words"),
    ("uniform_not_open", "return ((double)x + 0.5) * (1.0 / 4294967296.0);",
     "return ((double)x + 1.0) * (1.0 / 4294967296.0);",
     "test_oracle_noise.py::test_uniform_open_interval_endpoints"),
    # Box-Muller normals for the random displacement of Eq. 1
    ("box_muller_radius", "const double rho = sqrt(-2.0 * log(ora_uniform21(m[2 * k])));",
     "const double rho = sqrt(-log(ora_uniform21(m[2 * k])));",
     "test_oracle_noise.py::test_normals_are_standard_normal"),
    ("box_muller_reused_angle", "z[2 * k + 1] = rho * sin(theta);", "z[2 * k + 1] = rho * cos(theta);",
     "test_oracle_noise.py::test_replica_pairs_share_one_philox_output_as_three_box_muller_pairs"),
    ("replica_pair_same_half", "for (int d = 0; d < 3; ++d) xi[d] = z[3 * second + d];",
     "for (int d = 0; d < 3; ++d) xi[d] = z[d];",
     "test_oracle_noise.py::test_replica_pairs_share_one_philox_output_as_three_box_muller_pairs"),
    ("uniform21_radius_field_reused", "((x[0] & 0x7FFu) << 10) | (x[1] & 0x3FFu),",
     "x[0] >> 11,",
     "test_oracle_noise.py::test_replica_pairs_share_one_philox_output_as_three_box_muller_pairs"),
    ("exp1_sign", "return -log(ora_uniform(x[0]));", "return log(ora_uniform(x[0]));",
     "test_oracle_noise.py::test_exp1_thresholds_are_unit_exponential"),
    # spring laws
    ("fene_dropped_H", "double s = 1.0 - H * q2 / b;", "double s = 1.0 - q2 / b;",
     "test_oracle_model.py::test_fene_force_is_gradient_of_potential"),
    ("harmonic_not_unit_vector", "coef = q > 0.0 ? H * (q - r0) / q : 0.0;", "coef = q > 0.0 ? H * (q - r0) : 0.0;",
     "test_oracle_collapsed.py::test_zero_noise_step_moves_beads_down_the_potential_gradient"),
    ("vwf_constants_swapped", "f = ch->vwf_fb * x + ch->vwf_fa * x / s;", "f = ch->vwf_fa * x + ch->vwf_fb * x / s;",
     "test_oracle_vwf.py::test_zero_noise_step_is_minus_grad_u"),
    ("vwf_disulfide_reacts", "return ch->spring != ORA_SPRING_VWF || i % 2 == 0;", "return 1;",
     "test_oracle_vwf.py::test_only_a2_domains_unfold"),
    # Lennard-Jones cohesion (Sec. II)
    ("lj_factor", "const double dUdr_over_r = 12.0 * ch->lj_u * (x6 - x6 * x6) / rr;",
     "const double dUdr_over_r = 6.0 * ch->lj_u * (x6 - x6 * x6) / rr;",
     "test_oracle_collapsed.py::test_zero_noise_step_moves_beads_down_the_potential_gradient"),
    ("lj_includes_bonded_neighbours", "for (int j = i + 2; j < N; ++j) {", "for (int j = i + 1; j < N; ++j) {",
     "test_oracle_collapsed.py::test_zero_noise_step_moves_beads_down_the_potential_gradient"),
    ("vwf_odd_springs_are_a2", "if (i % 2 == 0) {\n        double s = 1.0 - x * x / (ch->vwf_xmax * ch->vwf_xmax);",
     "if (i % 2 == 1) {\n        double s = 1.0 - x * x / (ch->vwf_xmax * ch->vwf_xmax);",
     "test_oracle_vwf.py::test_zero_noise_step_is_minus_grad_u"),
    # Eq. 1 (free draining) and the flows
    ("diffusivity", "const double D = 0.25, kT = 1.0;\n    const int N = ch->n_beads;\n    double kappa[9];\n    ora_flow_gradient",
     "const double D = 0.5, kT = 1.0;\n    const int N = ch->n_beads;\n    double kappa[9];\n    ora_flow_gradient",
     "test_oracle_model.py::test_free_bead_noise_amplitude"),
    ("spring_reaction_sign", "if (i > 0)     fb -= F[3 * (i - 1) + d];", "if (i > 0)     fb += F[3 * (i - 1) + d];",
     "test_oracle_model.py::test_zero_noise_rouse_modes_decay_exactly"),
    ("shear_transposed", "case ORA_FLOW_SHEAR:    kappa[0 * 3 + 2] = rate; break;",
     "case ORA_FLOW_SHEAR:    kappa[2 * 3 + 0] = rate; break;",
     "test_oracle_model.py::test_shear_advection_direction"),
    # RPY tensor (Eqs. 2-3), its factor and the HI step
    ("rpy_far_coefficient", "cd = pre * (1.0 - 2.0 * a * a / rr);", "cd = pre * (1.0 - 2.0 * a * a / (3.0 * rr));",
     "test_oracle_hi.py::test_contact_mobilities"),
    ("rpy_overlap_coefficient", "ci = pre * (r / (2.0 * a)) * (8.0 / 3.0 - 3.0 * r / (4.0 * a));",
     "ci = pre * (r / (2.0 * a)) * (8.0 / 3.0 - 3.0 * r / (8.0 * a));",
     "test_oracle_hi.py::test_divergence_free"),
    ("noise_transposed_factor",
     "for (int q = 0; q <= p; ++q) noise[p] += Lc[p * n + q] * xi[q];",
     "for (int q = p; q < n; ++q) noise[p] += Lc[q * n + p] * xi[q];",
     "test_oracle_hi.py::test_noise_covariance_is_2_D_dt"),
    ("cholesky_wrong_row", "for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];",
     "for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[i * n + k];",
     "test_oracle_hi.py::test_tensor_positive_definite_and_factor"),
    ("rpy_diagonal_block", "for (int k = 0; k < 9; ++k) blk[k] = (k % 4 == 0) ? 1.0 : 0.0;",
     "for (int k = 0; k < 9; ++k) blk[k] = (k % 4 == 0) ? 0.75 : 0.0;",
     "test_oracle_hi.py::test_vanishing_radius_is_free_draining"),
    ("hi_drift_without_mobility", "for (int q = 0; q < n; ++q) drift[p] += W[p * n + q] * Fb[q];",
     "for (int q = 0; q < n; ++q) drift[p] += (p == q ? 1.0 : 0.0) * Fb[q];",
     "test_oracle_hi.py::test_zero_noise_drift_is_mobility_times_force"),
    # the estimator and the kinetics
    ("rsf_counts_the_parent", "const double fr = rsum[i] / R;", "const double fr = rsum[i] / (R + 1);",
     "test_oracle_method.py::test_identical_noise_replicas_reproduce_parent"),
    ("bell_sign", "*lam += ch->k0 * exp(f * ch->dx) * dT;", "*lam += ch->k0 * exp(-f * ch->dx) * dT;",
     "test_oracle_method.py::test_bell_constant_force_survival_closed_form"),
    ("threshold_last_not_first", "if (thr_on && *first_thr < 0 && f >= ch->f_c) *first_thr = step;",
     "if (thr_on && f >= ch->f_c) *first_thr = step;",
     "test_oracle_method.py::test_threshold_events_recount_from_window_profiles"),
    ("tsf_normalisation", "const double ft = tsum[i] / S;", "const double ft = tsum[i] / (S + 1);",
     "test_oracle_method.py::test_run_matches_procedure_written_out"),
    ("isf_interval", "(p->bell_mask >> ORA_ISF) & 1, ch, f[i], p->dt,",
     "(p->bell_mask >> ORA_ISF) & 1, ch, f[i], S * p->dt,",
     "test_oracle_method.py::test_bell_isf_hazard_at_equilibrium_matches_quadrature"),
    ("replica_noise_step_offset",
     "(uint32_t)(t + s), cid, &xi[3 * i]);\n                    nover += ora_em_step(ch, p->dt, p->s_min, rk, xi);",
     "(uint32_t)(t + s + 1), cid, &xi[3 * i]);\n                    nover += ora_em_step(ch, p->dt, p->s_min, rk, xi);",
     "test_oracle_method.py::test_identical_noise_replicas_reproduce_parent"),
    ("replicas_not_respawned",
     "double* rk = rep + 3 * (size_t)N * (k - 1);\n                memcpy(rk, parent, sizeof(double) * 3 * (size_t)N);",
     "double* rk = rep + 3 * (size_t)N * (k - 1);",
     "test_oracle_method.py::test_run_matches_procedure_written_out"),
    # Eq. 5 and R_GZ (Sec. III)
    ("eq5_laboratory_frame", "const double d = fabs((rk[3 * i + j] - ck[j]) - (parent[3 * i + j] - cp[j]));",
     "const double d = fabs(rk[3 * i + j] - parent[3 * i + j]);",
     "test_oracle_conformation.py::test_hookean_per_bead_difference_matches_exact_gaussian_expectation"),
    ("eq5_mean_over_springs", "dbar[(w * NR + repc_off[c] + k - 1) * 3 + j] = dsum[j] / N;",
     "dbar[(w * NR + repc_off[c] + k - 1) * 3 + j] = dsum[j] / (N - 1);",
     "test_oracle_conformation.py::test_two_beads_reduce_to_half_the_bond_change"),
    ("rgz_sample_variance", "return sqrt(s2 / N);", "return sqrt(s2 / (N - 1));",
     "test_oracle_conformation.py::test_rgz_of_a_straight_chain_along_z"),
    # the pathwise tangent
    ("tangent_db_sign", "*dc_db = -ch->H * ch->H * q2 / (ch->b * ch->b * s * s);",
     "*dc_db = ch->H * ch->H * q2 / (ch->b * ch->b * s * s);",
     "test_oracle_tangent.py::test_tangent_matches_common_random_number_finite_differences[1]"),
    ("force_tangent_dropped_factor",
     "const double dc = dcq * 2.0 * qdq + dcH * dH + dcb * db;\n    for (int d = 0; d < 3; ++d) dF[d]",
     "const double dc = dcq * qdq + dcH * dH + dcb * db;\n    for (int d = 0; d < 3; ++d) dF[d]",
     "test_oracle_tangent.py::test_tangent_matches_common_random_number_finite_differences[0]"),
    ("tension_tangent_dropped_division", "return dc * q + c * qdq / q;", "return dc * q + c * qdq;",
     "test_oracle_tangent.py::test_tangent_matches_common_random_number_finite_differences[0]"),
]


def _build(tmp, name, source):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    shutil.copy(os.path.join(ORACLE, "bd_oracle.h"), os.path.join(d, "bd_oracle.h"))
    with open(os.path.join(d, "bd_oracle.c"), "w") as fh:
        fh.write(source)
    lib = os.path.join(d, "libbdoracle_planted.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", lib,
                    os.path.join(d, "bd_oracle.c"), "-lm"], check=True)
    return lib


def _run_pins(lib, pins, extra=()):
    # one thread per pin process: the cases run side by side
    env = dict(os.environ, BD_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *extra,
                           *[os.path.join(ROOT, "tests", p) for p in pins]], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def planted_results(tmp_path_factory):
    """Every planted case compiled and its pin run, in parallel: name -> (returncode, output)."""
    src = open(os.path.join(ORACLE, "bd_oracle.c")).read()
    tmp = str(tmp_path_factory.mktemp("planted"))

    def one(case):
        name, orig, planted, pin = case
        if src.count(orig) != 1:
            return name, (None, f"the original text occurs {src.count(orig)} times")
        r = _run_pins(_build(tmp, name, src.replace(orig, planted)), [pin], extra=("-x",))
        return name, (r.returncode, (r.stdout + r.stderr)[-2000:])

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return dict(ex.map(one, PLANTED))


@pytest.mark.parametrize("name,pin", [(p[0], p[3]) for p in PLANTED], ids=[p[0] for p in PLANTED])
def test_planted_mistake_fails_its_pin(planted_results, name, pin):
    rc, out = planted_results[name]
    assert rc is not None, f"{name}: {out}"
    # exit code 1: the pin ran and failed (not a collection or usage error)
    assert rc == 1 and " failed" in out, f"{name}: {pin} did not catch it\n{out}"


def test_unplanted_copy_passes_the_pins(tmp_path):
    # the control: a copy built and loaded the same way, without a mistake, passes
    lib = _build(str(tmp_path), "control", open(os.path.join(ORACLE, "bd_oracle.c")).read())
    r = _run_pins(lib, sorted({p[3] for p in PLANTED}))
    assert r.returncode == 0, (r.stdout + r.stderr)[-2000:]
    assert " passed" in r.stdout and " failed" not in r.stdout
