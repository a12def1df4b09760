"""Planted mistakes in copies of the oracle must each fail at least one pin (CPU).

Each mutant is a textual edit of ``oracle/pasfm_oracle.c`` compiled into a
temporary directory; the oracle package is pointed at it for the duration of
the check and restored afterwards.  The committed oracle is never modified.
"""
import os
import subprocess

import pytest

import oracle
from tests import oracle_checks as oc

SRC = os.path.join(os.path.dirname(oracle.__file__), "pasfm_oracle.c")

MUTANTS = {
    "pulse_sign_flipped": ("return (prim(g, wh) - prim(g, wl)) / (2.0 * d * h);",
                           "return (prim(g, wl) - prim(g, wh)) / (2.0 * d * h);"),
    "pulse_amplitude_drops_1_over_d": ("return (prim(g, wh) - prim(g, wl)) / (2.0 * d * h);",
                                       "return (prim(g, wh) - prim(g, wl)) / (2.0 * 10.0 * h);"),
    "sample_time_off_by_half": ("const double tau = g->c * (g->t0 + (double)n / g->fs);\n  if",
                                "const double tau = g->c * (g->t0 + ((double)n + 0.5) / g->fs);\n  if"),
    "derivative_drops_W_over_d": ("return (dh - dl) / (2.0 * d * h) - W / d;",
                                  "return (dh - dl) / (2.0 * d * h);"),
    "derivative_sign_flipped": ("return (dh - dl) / (2.0 * d * h) - W / d;",
                                "return (dl - dh) / (2.0 * d * h) - W / d;"),
    "rotation_transposed": ("x[a] = P[4 * a] * e[0] + P[4 * a + 1] * e[1] + P[4 * a + 2] * e[2] + P[4 * a + 3];",
                            "x[a] = P[a] * e[0] + P[4 + a] * e[1] + P[8 + a] * e[2] + P[4 * a + 3];"),
    "voxel_axes_swapped": ("g->ox + g->dx * ix, g->oy + g->dy * iy, g->oz + g->dz * iz",
                           "g->ox + g->dx * iz, g->oy + g->dy * iy, g->oz + g->dz * ix"),
    "cross_product_sign": ("w[0] += x[1] * Gj[2] - x[2] * Gj[1];",
                           "w[0] += x[2] * Gj[1] - x[1] * Gj[2];"),
    "adjoint_reads_reversed_samples": ("for (int n = lo; n <= hi; ++n) acc += gs[n] * oracle_pulse(g, d, n);",
                                       "for (int n = lo; n <= hi; ++n) acc += gs[lo + hi - n] * oracle_pulse(g, d, n);"),
    "sample_range_too_narrow": ("double a = floor((d - rho - tau0) / h - 0.5) - 1.0;",
                                "double a = floor((d - rho - tau0) / h - 0.5) + 2.0;"),
    "pose_grad_ignores_mask": ("if (!mask || mask[fj]) {", "if (1) {"),
    # Gaussian kernel
    "gauss_prefactor_sigma_not_squared": ("if (g->kernel == 1) return g->sigma * g->sigma * exp(",
                                          "if (g->kernel == 1) return g->sigma * exp("),
    "gauss_antiderivative_width_doubled": (
        "return g->sigma * g->sigma * exp(-w * w / (2.0 * g->sigma * g->sigma));",
        "return g->sigma * g->sigma * exp(-w * w / (4.0 * g->sigma * g->sigma));"),
    "gauss_point_pulse_drops_amplitude_w": ("if (g->kernel == 1) return -w / (2.0 * d) * exp(",
                                            "if (g->kernel == 1) return -1.0 / (2.0 * d) * exp("),
    "gauss_derivative_drops_E": ("if (g->kernel == 1) return -w * exp(-w * w / (2.0 * g->sigma * g->sigma));",
                                 "if (g->kernel == 1) return -w;"),
    "gauss_support_two_sigma": ("return g->kernel == 1 ? 4.0 * g->sigma : g->a0;",
                                "return g->kernel == 1 ? 2.0 * g->sigma : g->a0;"),
}


def failing_pins():
    out = []
    if oc.check_closed_form() > 1e-12:
        out.append("closed_form")
    if oc.check_superposition() > 1e-12:
        out.append("superposition")
    if oc.check_adjoint_identity() > 1e-12:
        out.append("adjoint")
    if oc.check_rigid_invariance() > 1e-12:
        out.append("rigid")
    if oc.check_pulse_dd() > 1e-6:
        out.append("pulse_dd")
    if max(oc.check_pose_fd()) > 1e-6:
        out.append("pose_fd")
    if max(oc.check_pose_fd(use_mask=True, seed=11)) > 1e-6:
        out.append("pose_fd_masked")
    inside, outside = oc.check_wave_equation_gauss()
    if inside > 1e-8:
        out.append("gauss_wave_equation")
    if oc.check_quadrature_gauss() > 1e-9:
        out.append("gauss_quadrature")
    if oc.check_pulse_dd(gauss=True) > 1e-6:
        out.append("gauss_pulse_dd")
    if max(oc.check_pose_fd(sigma=0.06)) > 1e-6:
        out.append("gauss_pose_fd")
    return out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           str(csrc), "-o", str(so), "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle.load(str(so)))
    fails = failing_pins()
    assert fails, f"mutant {name} passed every pin"


# ----------------------------------------------------------------------------- TGV oracle (Python)

TGV_MUTANTS = {
    "transpose_sign": ("out[tuple(dst)] += y[tuple(src)]", "out[tuple(dst)] -= y[tuple(src)]"),
    "sym_gradient_drops_half": ("E[a, b] = 0.5 * (Dw[a][b] + Dw[b][a])", "E[a, b] = (Dw[a][b] + Dw[b][a])"),
    "w_gradient_drops_q": ("[-q[b] + sum(", "[sum("),
    "difference_not_scaled": ("out[tuple(lo)] = (v[tuple(hi)] - v[tuple(lo)]) / d",
                              "out[tuple(lo)] = (v[tuple(hi)] - v[tuple(lo)])"),
}


@pytest.mark.parametrize("name", sorted(TGV_MUTANTS))
def test_tgv_mutant_is_caught(name, monkeypatch):
    import importlib.util
    import sys

    import oracle.tgv as tgv_mod

    old, new = TGV_MUTANTS[name]
    src = open(tgv_mod.__file__).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    spec = importlib.util.spec_from_loader("oracle.tgv", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src.replace(old, new), tgv_mod.__file__, "exec"), mod.__dict__)
    monkeypatch.setitem(sys.modules, "oracle.tgv", mod)
    monkeypatch.setattr(oracle, "tgv", mod, raising=False)
    fails = [n for n, bad in (("sparse", oc.check_tgv_sparse() > 1e-12), ("fd", oc.check_tgv_fd() > 1e-7),
                               ("constant", oc.check_tgv_constant() > 1e-14)) if bad]
    assert fails, f"TGV mutant {name} passed every pin"


# ----------------------------------------------------------------------------- Adam and retraction (Python)

ADAM_MUTANTS = {
    # (module, old, new)
    "betas_swapped": ("adam", "m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * grad\n",
                      "m = b2 * np.asarray(m, dtype=np.float64) + (1 - b2) * grad\n"),
    "second_moment_of_g_not_g2": ("adam", "v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * grad * grad\n",
                                  "v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * np.abs(grad)\n"),
    "no_bias_correction_of_m": ("adam", "mh = m / (1 - b1 ** k)\n    vh = v / (1 - b2 ** k)\n    out",
                                "mh = m\n    vh = v / (1 - b2 ** k)\n    out"),
    "bias_correction_fixed_at_step_1": ("adam", "mh = m / (1 - b1 ** k)\n    vh = v / (1 - b2 ** k)\n    out",
                                        "mh = m / (1 - b1)\n    vh = v / (1 - b2)\n    out"),
    "pose_betas_swapped": ("adam", "m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * grad6",
                           "m = b2 * np.asarray(m, dtype=np.float64) + (1 - b2) * grad6"),
    "pose_rates_swapped": ("adam", "lr = np.array([lr_rot] * 3 + [lr_trans] * 3)",
                           "lr = np.array([lr_trans] * 3 + [lr_rot] * 3)"),
    "fixed_frame_moments_not_updated": ("adam", "        if fixed is not None and fixed[f]:\n            continue\n",
                                        "        if fixed is not None and fixed[f]:\n            m[f] = 0.0\n"
                                        "            continue\n"),
    "retraction_on_the_right": ("rigid", "out[:, :3] = E @ pose[:, :3]", "out[:, :3] = pose[:, :3] @ E"),
    "translation_not_rotated": ("rigid", "out[:, 3] = E @ pose[:, 3] + xi[3:]", "out[:, 3] = pose[:, 3] + xi[3:]"),
}

ADAM_PINS = ["test_adam_first_step_is_signed_lr", "test_adam_pose_first_step_moves_by_signed_lr",
             "test_adam_constant_gradient_steps_by_lr_every_step", "test_adam_alternating_gradient_closed_form",
             "test_adam_gradient_then_zero_separates_the_betas",
             "test_adam_pose_moments_follow_the_same_closed_forms", "test_retraction_closed_forms",
             "test_adam_pose_fixed_frame_keeps_pose_but_updates_moments"]


@pytest.mark.parametrize("name", sorted(ADAM_MUTANTS))
def test_adam_mutant_is_caught(name, monkeypatch):
    import importlib

    from tests import test_oracle_pins as pins

    modname, old, new = ADAM_MUTANTS[name]
    mod = importlib.import_module(f"oracle.{modname}")
    src = open(mod.__file__).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    mut = type(mod)(mod.__name__)
    mut.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mut.__dict__)
    if modname == "rigid":
        # adam_poses retracts through rigid.apply_twist: give it the mutated one too
        monkeypatch.setattr(pins.adam, "apply_twist", mut.apply_twist)
    monkeypatch.setattr(pins, modname, mut)
    fails = []
    for t in ADAM_PINS:
        try:
            getattr(pins, t)()
        except AssertionError:
            fails.append(t)
    assert fails, f"Adam mutant {name} passed every pin"
