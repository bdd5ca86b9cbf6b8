"""The oracle's pins have teeth: plant a plausible mistake in a copy of the
oracle's C source, compile it, point the oracle at it, and require that at
least one pin of tests/test_oracle_pins.py fails.  Each mutant is the kind of
slip a transcription of the force law, its adjoint, the binning or the lists
could contain.  All on the CPU (the mistakes are planted in the oracle only).
"""

import ctypes
import os
import subprocess
import types

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_sks_pins as sks_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "hacc_oracle.c")
SKS_SRC = os.path.join(os.path.dirname(oracle.__file__), "sks.py")

# (name, text in the oracle source, replacement)
MUTANTS = [
    ("softening dropped", "return pow(s + eps, -1.5) - poly5(c, s);", "return pow(s, -1.5) - poly5(c, s);"),
    ("pair vector reversed", "d[0] = min_image(x[j] - xi, L);", "d[0] = min_image(xi - x[j], L);"),
    ("force pair vector reversed", "double dx = min_image(x[j] - xi, L);", "double dx = min_image(xi - x[j], L);"),
    ("source mass swapped", "double g = m[j] * ora_fsr(s, eps, c);", "double g = m[i] * ora_fsr(s, eps, c);"),
    ("polynomial index", "s * (c[4] + s * c[5])", "s * (c[4] + s * c[4])"),
    ("polynomial sign", "return pow(s + eps, -1.5) - poly5(c, s);", "return pow(s + eps, -1.5) + poly5(c, s);"),
    ("no periodic image", "return d - L * nearbyint(d / L);", "return d;"),
    ("cutoff not strict", "if (!(s < rc2)) continue;\n            double g", "if (!(s <= rc2)) continue;\n            double g"),
    ("cutoff radius not squared", "double rc2 = rcut * rcut;\n#pragma omp parallel for schedule(dynamic, 4)\n    for (int64_t t = 0; t < S; ++t) {\n        int64_t i = targets[t];\n        double xi",
     "double rc2 = rcut;\n#pragma omp parallel for schedule(dynamic, 4)\n    for (int64_t t = 0; t < S; ++t) {\n        int64_t i = targets[t];\n        double xi"),
    ("derivative exponent", "return -1.5 * pow(s + eps, -2.5) - dpoly5(c, s);",
     "return -1.5 * pow(s + eps, -1.5) - dpoly5(c, s);"),
    ("adjoint factor 2 dropped", "double Jlj = f * lj[a] + 2.0 * fp * d[a] * dlj;",
     "double Jlj = f * lj[a] + fp * d[a] * dlj;"),
    ("adjoint own-term mass", "g[a] += mi * Jlj - mj * Jli;", "g[a] += mj * Jlj - mj * Jli;"),
    ("mass gradient sign", "gmi += -f * dlj;", "gmi += f * dlj;"),
    ("unstable placement", "for (int64_t i = 0; i < N; ++i) {\n        int64_t k = cnt[cell_of[i]]++;",
     "for (int64_t i = N - 1; i >= 0; --i) {\n        int64_t k = cnt[cell_of[i]]++;"),
    ("wrap correction dropped", "    if (xw >= L) xw = xw - L;\n    return xw;", "    return xw;"),
    ("cell key axes swapped", "int32_t c = (cz * n + cy) * n + cx;", "int32_t c = (cx * n + cy) * n + cz;"),
    ("float64 wrap correction dropped", "    if (pw >= L) pw = pw - L;\n    return pw;", "    return pw;"),
    ("displaced position rounded before the offset", "*o = (float)(pw - (double)ctr);", "*o = (float)pw - ctr;"),
    ("stencil row missing", "for (int dz = -R; dz <= R; ++dz)", "for (int dz = -R; dz < R; ++dz)"),
    ("image shift sign", "if (px < 0) { px += n; sx = -1; }", "if (px < 0) { px += n; sx = 1; }"),
    ("cell origin offset", "float ctr = ((float)c + 0.5f) * w;\n        *o = xw - ctr;",
     "float ctr = ((float)c + 1.5f) * w;\n        *o = xw - ctr;"),
    ("potential sign", "return (1.0 / sqrt(rc2 + eps) + 0.5 * P6(c, rc2)) - (1.0 / sqrt(s + eps) + 0.5 * P6(c, s));",
     "return (1.0 / sqrt(rc2 + eps) + 0.5 * P6(c, rc2)) - (1.0 / sqrt(s + eps) - 0.5 * P6(c, s));"),
    ("potential polynomial index", "s * (c[4] / 5.0 + s * c[5] / 6.0)", "s * (c[4] / 5.0 + s * c[5] / 5.0)"),
    ("rcb axis: shortest side", "if (hi[a] - lo[a] > hi[axis] - lo[axis]) axis = a;",
     "if (hi[a] - lo[a] < hi[axis] - lo[axis]) axis = a;"),
    ("rcb strict split", "int left = S->q[3 * i + axis] <= split;", "int left = S->q[3 * i + axis] < split;"),
    ("rcb mean rounded up", "int64_t split = sum[axis] / cnt;", "int64_t split = (sum[axis] + cnt - 1) / cnt;"),
    ("rcb unstable partition", "for (int64_t i = b; i < e; ++i) {\n                int left",
     "for (int64_t i = e - 1; i >= b; --i) {\n                int left"),
    ("rcb leaf size off by one", "if (cnt <= S->leaf_max || depth", "if (cnt < S->leaf_max || depth"),
    ("rcb image shift sign", "double jlo = (double)(leaf_qbox[6 * j + a] - 1) * scale + (double)sh[a] * (double)L;",
     "double jlo = (double)(leaf_qbox[6 * j + a] - 1) * scale - (double)sh[a] * (double)L;"),
    ("list gap off by one", "double gx = abs(dx) > 1 ? (double)(abs(dx) - 1) : 0.0;",
     "double gx = abs(dx) > 2 ? (double)(abs(dx) - 2) : 0.0;"),
    ("list predicate not strict", "return (gx * gx + gy * gy + gz * gz) * w * w < rc * rc;",
     "return (gx * gx + gy * gy + gz * gz) * w * w <= rc * rc;"),
    ("rcb boxes widened twice", "double ilo = (double)(leaf_qbox[6 * i + a] - 1) * scale;",
     "double ilo = (double)(leaf_qbox[6 * i + a] - 2) * scale;"),
    ("rcb lists not strict", "if (d2 < rc2) {", "if (d2 <= rc2) {"),
    ("drift before kick", "        vx[i] += dt_k * ax[i];\n        vy[i] += dt_k * ay[i];\n        vz[i] += dt_k * az[i];\n        if (x) {\n            x[i] += dt_d * vx[i];",
     "        if (x) x[i] += dt_d * vx[i];\n        vx[i] += dt_k * ax[i];\n        vy[i] += dt_k * ay[i];\n        vz[i] += dt_k * az[i];\n        if (x) {\n            x[i] += 0.0;"),
]

# the pins, fastest first (a mutant stops at its first failing pin)
PINS = [
    pins.test_kick_drift_exact_on_dyadic_values,
    pins.test_softened_newton_closed_form,
    pins.test_newton_limit_inverse_square,
    pins.test_polynomial_term_matches_numpy_polyval,
    pins.test_cutoff_is_exact_zero_and_strict,
    pins.test_periodic_image_across_boundary,
    pins.test_superposition_and_mass_linearity,
    pins.test_brute_force_small_against_independent_numpy,
    pins.test_perfect_lattice_has_zero_force,
    pins.test_newton_third_law_and_translation_invariance,
    pins.test_potential_closed_form_and_cutoff,
    pins.test_force_is_minus_gradient_of_potential_energy,
    pins.test_adjoint_against_finite_differences,
    pins.test_adjoint_against_torch_float64_autograd,
    pins.test_binning_invariants_and_numpy_restatement,
    pins.test_binning_with_displacements_keeps_float64_positions,
    lambda: pins.test_lists_cover_every_pair_within_cutoff(16.0, 3.0, 3.0),
    lambda: pins.test_lists_are_exactly_the_cells_whose_boxes_come_closer_than_rc(9.0, 1.0, 3.0),
    lambda: pins.test_lists_are_exactly_the_cells_whose_boxes_come_closer_than_rc(6.4, 0.375, 3.0),
    pins.test_rcb_hand_worked_examples,
    pins.test_rcb_regular_lattice_is_bit_interleaved,
    pins.test_rcb_leaves_invariants_on_clustered_particles,
    lambda: pins.test_rcb_lists_cover_every_pair_within_cutoff("uniform", 16),
    lambda: pins.test_rcb_lists_cover_every_pair_within_cutoff("clustered", 24),
    lambda: pins.test_rcb_lists_are_exactly_the_leaves_whose_widened_boxes_come_closer("uniform", 16),
    pins.test_rcb_lists_cutoff_is_strict_on_exact_gaps,
    pins.test_trajectory_gradient_against_finite_differences,
]


def _build(src_text, out_dir, tag):
    c_path = os.path.join(out_dir, f"mut_{tag}.c")
    so_path = os.path.join(out_dir, f"libmut_{tag}.so")
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                           "-o", so_path, c_path, "-lm"])
    return oracle.configure(ctypes.CDLL(so_path))


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    survivors = []
    saved = oracle.lib()
    try:
        for k, (name, old, new) in enumerate(MUTANTS):
            assert src.count(old) >= 1, f"mutation site not found: {name}"
            oracle._lib = _build(src.replace(old, new, 1), str(tmp_path), k)
            caught = False
            for pin in PINS:
                try:
                    pin()
                except Exception:  # an assertion, or a numerical blow-up the mistake causes
                    caught = True
                    break
            if not caught:
                survivors.append(name)
    finally:
        oracle._lib = saved
    assert not survivors, f"mistakes no pin catches: {survivors}"


def test_unmutated_oracle_passes_every_pin():
    for pin in PINS:
        pin()


# Planted mistakes in the sub-cycle reference (oracle/sks.py): the order and
# length of the half-streams and the kick, the wrap, the energy factors.
_S1 = "x = np.mod(x + 0.5 * h * v, L)\n        a = sr_force(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)"
_K = "v = v + h * a\n        x = np.mod(x + 0.5 * h * v, L)\n        hist"
SKS_MUTANTS = [
    ("first stream by a full step", _S1, _S1.replace("0.5 * h * v", "h * v")),
    ("force before the first stream", _S1,
     "a = sr_force(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)\n        x = np.mod(x + 0.5 * h * v, L)"),
    ("kick-stream-kick instead of stream-kick-stream", _S1 + "\n        " + _K,
     "a = sr_force(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)\n        v = v + 0.5 * h * a\n"
     "        x = np.mod(x + h * v, L)\n        a = sr_force(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)\n"
     "        v = v + 0.5 * h * a\n        hist"),
    ("second stream with the old velocity", _K,
     "x = np.mod(x + 0.5 * h * v, L)\n        v = v + h * a\n        hist"),
    ("kick by half a step", _K, _K.replace("v = v + h * a", "v = v + 0.5 * h * a")),
    ("final stream not wrapped", _K, _K.replace("x = np.mod(x + 0.5 * h * v, L)", "x = x + 0.5 * h * v")),
    ("kinetic energy without the half", "0.5 * np.sum(m[:, None] * v * v)", "np.sum(m[:, None] * v * v)"),
    ("pair potential counted twice", "0.5 * np.sum(m * phi)", "np.sum(m * phi)"),
]


def _sks_module(src_text):
    mod = types.ModuleType("oracle._sks_mutant")
    mod.__package__ = "oracle"
    exec(compile(src_text, "sks_mutant.py", "exec"), mod.__dict__)
    return mod


def test_every_planted_subcycle_mistake_fails_a_pin():
    src = open(SKS_SRC).read()
    survivors = []
    for name, old, new in SKS_MUTANTS:
        assert src.count(old) == 1, f"mutation site not found: {name}"
        mod = _sks_module(src.replace(old, new, 1))
        caught = False
        for check in sks_pins.SKS_CHECKS:
            try:
                check(mod)
            except Exception:
                caught = True
                break
        if not caught:
            survivors.append(name)
    assert not survivors, f"sub-cycle mistakes no pin catches: {survivors}"


def test_unmutated_subcycles_pass_every_pin():
    mod = _sks_module(open(SKS_SRC).read())
    for check in sks_pins.SKS_CHECKS:
        check(mod)
