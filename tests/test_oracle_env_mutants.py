"""The pins of the environment, particle-filter and neural-network oracle
(utrack_oracle.c, utrack_oracle_nn.c) catch plausible mistakes: for each
planted mistake a copy of the oracle's C sources is made
with that one edit, the oracle module is pointed at it (UTRACK_ORACLE_DIR)
in a child process, and the pin tests named for it must fail there; an
unmodified copy passes the same tests (the control case)."""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
SOURCES = ("utrack_oracle.c", "utrack_oracle_nn.c", "utrack_oracle_ppo.c")

E, P, R = "tests/test_oracle_env.py", "tests/test_oracle_pf.py", "tests/test_oracle_rng.py"
N = "tests/test_oracle_nn.py"

# name: (file, exact source text, replacement, pin tests that must catch it)
MUTANTS = {
    "kinematics_sin_for_cos": ("utrack_oracle.c", "s->ax[i] += c->agent_speed * c->dt * cos(psi);",
                               "s->ax[i] += c->agent_speed * c->dt * sin(psi);",
                               [E + "::test_straight_line_closed_form"]),
    "target_step_drops_dt": ("utrack_oracle.c", "s->tx[j] += s->tspeed[j] * c->dt * cos(psi);",
                             "s->tx[j] += s->tspeed[j] * cos(psi);", [E + "::test_targets_drift_free_is_straight"]),
    "detection_radius_halved": ("utrack_oracle.c", "valid[q] = d <= c->det_radius;",
                                "valid[q] = d <= 0.5 * c->det_radius;",
                                [E + "::test_noise_free_ranges_equal_distance_and_detection_edge"]),
    "comms_radius_inverted": ("utrack_oracle.c", "sqrt(dx * dx + dy * dy) <= c->comm_radius",
                              "sqrt(dx * dx + dy * dy) >= c->comm_radius", [E + "::test_comms_brute_force"]),
    "velocity_cap_doubled": ("utrack_oracle.c", "if (sp > c->pf_vcap) {", "if (sp > 2.0 * c->pf_vcap) {",
                             [P + "::test_velocity_cap"]),
    "likelihood_variance_halved": ("utrack_oracle.c", "- acc / (2.0 * c->range_sigma * c->range_sigma);",
                                   "- acc / (c->range_sigma * c->range_sigma);",
                                   [P + "::test_weights_brute_force_bayes_p4"]),
    "resample_tie_rule": ("utrack_oracle.c", "while ((int64_t)P * Q[i] <= thr) ++i;",
                          "while ((int64_t)P * Q[i] < thr) ++i;", [P + "::test_resample_brute_force_small"]),
    "reward_exponent_factor": ("utrack_oracle.c", "return exp(-2.0 * t / (1.0 - t));",
                               "return exp(-t / (1.0 - t));", [E + "::test_tracking_reward_eq1_printed_values"]),
    "crash_never_set": ("utrack_oracle.c", "if (sqrt(dx * dx + dy * dy) < c->d_safe) cr = 1;",
                        "if (sqrt(dx * dx + dy * dy) < c->d_safe) cr = 0;",
                        [E + "::test_reward_follow_normalisation_and_crash"]),
    "philox_multiplier": ("utrack_oracle.c", "uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
                          "uint64_t prod0 = (uint64_t)0xD2511F55u * (uint64_t)c0;",
                          [R + "::test_philox_is_invertible_round_function"]),
    "ls_normal_equation_factor": ("utrack_oracle.c", "b0 += 0.5 * dx * da;", "b0 += dx * da;",
                                  ["tests/test_oracle_ls.py::test_exact_static_target_from_noise_free_ranges"]),
    "ls_solve_sign": ("utrack_oracle.c", "ey = e1y + (a00 * b1 - a01 * b0) / det;",
                      "ey = e1y + (a00 * b1 + a01 * b0) / det;",
                      ["tests/test_oracle_ls.py::test_exact_static_target_from_noise_free_ranges"]),
    "ess_trigger_inverted": ("utrack_oracle.c",
                             "resample = resample && 16u * s1 * s1 < (uint64_t)c->pf_ess_num * (uint64_t)P * s2;",
                             "resample = resample && 16u * s1 * s1 > (uint64_t)c->pf_ess_num * (uint64_t)P * s2;",
                             ["tests/test_oracle_ess.py::test_trigger_is_the_integer_rule_on_the_weights"]),
    "ess_carried_weights_unshifted": ("utrack_oracle.c",
                                      "s->pw[(int64_t)f * P + i] = resample ? 0.0 : l[i] - lmax;",
                                      "s->pw[(int64_t)f * P + i] = resample ? 0.0 : l[i];",
                                      ["tests/test_oracle_ess.py::test_carried_weights_are_the_product_of_likelihoods"]),
    "token_kind_flags_swapped": ("utrack_oracle.c", "        t[5] = 1.0;\n        slot++;",
                                 "        t[4] = 1.0;\n        slot++;", [E + "::test_observation_tokens_structure"]),
    "estimate_motion_smoothing": ("utrack_oracle.c", "#define OC_VEL_KEEP 0.85", "#define OC_VEL_KEEP 0.8",
                                  [P + "::test_estimate_motion_features_closed_form"]),
    "critic_token_velocity_sin_cos": ("utrack_oracle_ppo.c",
                                      "q[3] = agent_speed * cos(apsi[a]); q[4] = agent_speed * sin(apsi[a]);",
                                      "q[3] = agent_speed * sin(apsi[a]); q[4] = agent_speed * cos(apsi[a]);",
                                      ["tests/test_oracle_ppo.py::test_state_token_velocities_are_the_next_displacement"]),
    # the transformer agent, the estimator MLP and Adam (utrack_oracle_nn.c)
    "agent_attention_scale_lost": ("utrack_oracle_nn.c", "att[s] = acc / sqrt((double)dh);", "att[s] = acc;",
                                   [N + "::test_policy_matches_torch_encoder"]),
    "agent_layernorm_epsilon": ("utrack_oracle_nn.c", "double inv = 1.0 / sqrt(var + 1e-5);",
                                "double inv = 1.0 / sqrt(var + 1e-3);", [N + "::test_policy_matches_torch_encoder"]),
    "mlp_gelu_derivative_lost": ("utrack_oracle_nn.c", "dz[j] = da[j] * gelu_grad(z[j]);", "dz[j] = da[j];",
                                 [N + "::test_mlp_grad_central_differences"]),
    "huber_slope_sign": ("utrack_oracle_nn.c", "*drho = e > 0.0 ? delta : -delta;", "*drho = delta;",
                         [N + "::test_mlp_huber_matches_torch_huber_loss"]),
    "adam_second_moment_decay": ("utrack_oracle_nn.c", "v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];",
                                 "v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i];", [N + "::test_adam_matches_torch"]),
}


def _copy(dst, edit=None):
    os.makedirs(dst, exist_ok=True)
    for name in SOURCES:
        text = open(os.path.join(ORACLE, name)).read()
        if edit and edit[0] == name:
            assert text.count(edit[1]) == 1, f"mutation site not unique in {name}: {edit[1]}"
            text = text.replace(edit[1], edit[2])
        with open(os.path.join(dst, name), "w") as f:
            f.write(text)


def _run(src_dir, tests):
    env = dict(os.environ, UTRACK_ORACLE_DIR=src_dir)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"] + tests
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def workdir():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tempfile.mkdtemp()
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmodified_copy_passes_the_pins(workdir):
    d = os.path.join(workdir, "control")
    _copy(d)
    tests = sorted({t for m in MUTANTS.values() for t in m[3]})
    r = _run(d, tests)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_its_pins(name, workdir):
    fname, old, new, tests = MUTANTS[name]
    d = os.path.join(workdir, name)
    _copy(d, (fname, old, new))
    r = _run(d, tests)
    assert r.returncode != 0, f"{name} passed {tests}"
    assert "failed" in r.stdout or "error" in r.stdout.lower(), r.stdout[-1000:]
