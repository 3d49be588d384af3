"""The oracle's pins against planted mistakes (mutation testing, CPU only).

Each mutant is a copy of the oracle's sources with one plausible mistake
planted by a textual replacement that matches exactly once: a dropped term,
a wrong sign, a wrong index, a transposed operand, a swapped shape function
or weight.  The copy is compiled with the oracle's own flags into a
temporary library, and the pin tests of that part of the oracle are run
against it in a subprocess (the oracle package is pointed at the copy before
its first call).  Every mutant must make at least one pin fail; the
unmutated copy, built and run the same way, must pass them all.

The Python parts (the PTA loop, the block front end) are mutated the same
way in a copy of the package that the subprocess imports first.  Tests that
compare the product with the oracle are left out of these runs: a mistake
caught only there would be caught by the product, not by a pin.

Mutants that cannot change any result are not listed: for instance the time
average weighted by a constant dt, or a boundary comparison that the inputs
never meet.  The committed oracle sources are only read; nothing here
changes them.
"""

import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
SOURCES = ["ptadd_oracle.c", "mlp_oracle.c", "junction_oracle.c"]
HEADER = "ptadd_oracle.h"

PINS = "tests/test_oracle_pins.py"
JPINS = "tests/test_junction_oracle.py"
MPINS = "tests/test_mlp_oracle.py"
PTAPINS = "tests/test_pta_oracle.py"
BLOCKPINS = "tests/test_blocks.py"
ALL_PINS = (PINS, JPINS, MPINS, PTAPINS, BLOCKPINS)
# tests of these files that compare the product with the oracle: a mistake
# caught only there is caught by the product, not pinned, so they do not run
DESELECT = {PTAPINS: "not product_pta_driver",
            BLOCKPINS: "not c_abi_block_functions_match and not block_driver_follows"}

# (name, source file, text, replacement, pin file)
MUTANTS = [
    # the segment stress (nonsingular isotropic field, Sec. 2.1)
    ("a2_term_dropped_in_A0", "ptadd_oracle.c",
     "const double A0 = 2.0 * J[0] + 3.0 * a2 * J[2];", "const double A0 = 2.0 * J[0];", PINS),
    ("sign_of_q_term_in_g", "ptadd_oracle.c",
     "G[i] = -(A0 * Rxb[i] + A1 * q[i]);", "G[i] = -(A0 * Rxb[i] - A1 * q[i]);", PINS),
    ("poisson_factor_sign", "ptadd_oracle.c",
     "mu / (4.0 * ORC_PI * (1.0 - nu))", "mu / (4.0 * ORC_PI * (1.0 + nu))", PINS),
    ("sign_of_the_J3_term", "ptadd_oracle.c",
     "- (Rp[al] * t[be] + t[al] * Rp[be]) * J[3]", "+ (Rp[al] * t[be] + t[al] * Rp[be]) * J[3]", PINS),
    ("diagonal_J2_dropped", "ptadd_oracle.c",
     "dab * qR * (J[0] + 3.0 * a2 * J[2])", "dab * qR * J[0]", PINS),
    ("J1_wrong_index", "ptadd_oracle.c",
     "J[1] = dr / (r1 * r2);", "J[1] = dr / (r1 * r1);", PINS),
    ("straddling_J0_sign", "ptadd_oracle.c",
     "J[0] = u2 / (d2 * r2) - u1 / (d2 * r1);", "J[0] = u2 / (d2 * r2) + u1 / (d2 * r1);", PINS),
    ("one_side_J2_tail_term", "ptadd_oracle.c",
     "return (w + 2.0 * r) / (3.0 * r * r * r * (r + w) * (r + w));",
     "return (w + r) / (3.0 * r * r * r * (r + w) * (r + w));", PINS),
    ("gauss_weights_swapped", "ptadd_oracle.c",
     "GL4_W[4] = {0.3478548451374538, 0.6521451548625461,",
     "GL4_W[4] = {0.6521451548625461, 0.3478548451374538,", PINS),
    # the Peach-Koehler force and the nodal assembly (Sec. 2.1)
    ("pk_force_operands_transposed", "ptadd_oracle.c",
     "cross3(sb, t, f);", "cross3(t, sb, f);", PINS),
    ("shape_function_swapped", "ptadd_oracle.c",
     "Fs[c] += L * w[q] * (1.0 - xi[q]) * f[c];", "Fs[c] += L * w[q] * xi[q] * f[c];", PINS),
    ("stress_times_b_index", "ptadd_oracle.c",
     "out[0] = s[0] * v[0] + s[5] * v[1] + s[4] * v[2];",
     "out[0] = s[0] * v[0] + s[4] * v[1] + s[5] * v[2];", PINS),
    ("nodal_assembly_neighbour", "ptadd_oracle.c",
     "FsFe[6 * prv[a] + 3 + c]", "FsFe[6 * nxt[a] + 3 + c]", PINS),
    ("subset_assembly_wrong_end", "ptadd_oracle.c",
     "F_out[3 * k + c] = Fs[c] + Ge[c];", "F_out[3 * k + c] = Fs[c] + Gs[c];", PINS),
    # the glide mobility (Eq. 2.1), lumped and consistent
    ("glide_projection_dropped", "ptadd_oracle.c",
     "v[c] = (Fa[c] - n[c] * nF) / (B * M);", "v[c] = Fa[c] / (B * M);", PINS),
    ("lumped_mass_not_halved", "ptadd_oracle.c",
     "const double M = 0.5 * (sqrt(dot3(dp, dp)) + sqrt(dot3(dn, dn)));",
     "const double M = (sqrt(dot3(dp, dp)) + sqrt(dot3(dn, dn)));", PINS),
    ("consistent_mass_off_diagonal", "ptadd_oracle.c",
     "A[i * m + j] += B * L / 6.0;", "A[i * m + j] += B * L / 3.0;", PINS),
    # the averages (Eq. 2.5), the polar velocity (Eq. 2.11) and the Euler step
    ("lp_outer_product_transposed", "ptadd_oracle.c",
     "acc[al * 3 + be] += bv[al] * c[be];", "acc[al * 3 + be] += bv[be] * c[al];", PINS),
    ("lp_cross_product_sign", "ptadd_oracle.c",
     "cross3(dx, vb, c);", "cross3(vb, dx, c);", PINS),
    ("rho_squared_length", "ptadd_oracle.c",
     "len += sqrt(dot3(dx, dx));", "len += dot3(dx, dx);", PINS),
    ("polar_velocity_length_dropped", "ptadd_oracle.c",
     "acc[m] += L * 0.5 * (v[3 * i + m] + v[3 * j + m]);",
     "acc[m] += 0.5 * (v[3 * i + m] + v[3 * j + m]);", PINS),
    ("euler_step_sign", "ptadd_oracle.c",
     "++m) x[m] += v[m] * dt;", "++m) x[m] -= v[m] * dt;", PINS),
    # the network tables, the total stress and the pinned nodes
    ("loop_left_open", "ptadd_oracle.c",
     "nxt[i] = (i + 1 < e) ? i + 1 : b;", "nxt[i] = (i + 1 < e) ? i + 1 : e - 1;", PINS),
    ("applied_stress_dropped", "ptadd_oracle.c",
     "for (int c = 0; c < 6; ++c) sig[c] = sig_app[c];", "for (int c = 0; c < 6; ++c) sig[c] = 0.0 * sig_app[c];", PINS),
    ("half_the_interactions", "ptadd_oracle.c",
     "for (int64_t i = 0; i < n_nodes; ++i) {\n        orc_seg_stress",
     "for (int64_t i = 0; i < n_nodes; i += 2) {\n        orc_seg_stress", PINS),
    ("pinned_nodes_move", "ptadd_oracle.c",
     "if ((pinned && pinned[a]) || !(M > 0.0)) {", "if (!(M > 0.0)) {", PINS),
    ("segments_skipped_at_one_pinned_end", "ptadd_oracle.c",
     "if (skip_pinned && pinned && pinned[i] && pinned[nxt[i]]) continue;",
     "if (skip_pinned && pinned && pinned[i]) continue;", PINS),
    # the brute-force reference the analytic field is checked against
    ("quadrature_reference_laplacian_sign", "ptadd_oracle.c",
     "(d3[(i * 3 + al) * 3 + be] - ((al == be) ? dl[i] : 0.0L))",
     "(d3[(i * 3 + al) * 3 + be] + ((al == be) ? dl[i] : 0.0L))", PINS),
    ("quadrature_reference_weight", "ptadd_oracle.c",
     "const long double wt = 0.5L * h * w[g];", "const long double wt = h * w[g];", PINS),
    # junctions (Sec. 2.2): the counter-based generator, the capture distance,
    # the release and the clock jump
    ("splitmix_shift", "junction_oracle.c",
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBull;", JPINS),
    ("break_fraction_counter", "junction_oracle.c",
     "(uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull", "(uint64_t)k * 0x9E3779B97F4A7C15ull", JPINS),
    ("far_end_not_clamped", "junction_oracle.c",
     "if (u > 1.0) u = 1.0;", "if (u > 2.0) u = 2.0;", JPINS),
    ("release_strictly_after_the_break", "junction_oracle.c",
     "jbreak[p] <= t) {", "jbreak[p] < t) {", JPINS),
    ("jump_from_the_step_start", "junction_oracle.c",
     "const double jump = tmin - t1;", "const double jump = tmin - t;", JPINS),
    ("held_node_keeps_moving", "junction_oracle.c",
     "v[3 * p] = v[3 * p + 1] = v[3 * p + 2] = 0.0;\n                held += 1;", "held += 1;", JPINS),
    ("recaptured_by_the_loop_it_left", "junction_oracle.c",
     "if (loop_of[q] == loop_of[p] || loop_of[q] == jlast[p]) continue;",
     "if (loop_of[q] == loop_of[p]) continue;", JPINS),
    ("capture_radius_doubled", "junction_oracle.c",
     "x + 3 * nxt[q]) < rc2) {", "x + 3 * nxt[q]) < 4.0 * rc2) {", JPINS),
    ("density_dropped_over_the_jump", "junction_oracle.c",
     "S_rho += rho * jump;", "S_rho += 0.0 * jump;", JPINS),
    ("pinned_rows_keep_their_coupling", "ptadd_oracle.c",
     "for (int64_t q = 0; q < m; ++q) A[i * m + q] = 0.0;\n                A[i * m + i] = 1.0;",
     "A[i * m + i] = 1.0;", PINS),
    # the surrogate's network (Sec. 3.3): activation, loss gradient, Adam
    ("gelu_derivative_exponent", "mlp_oracle.c",
     "z * exp(-0.5 * z * z) / sqrt(2.0 * pi)", "z * exp(-z * z) / sqrt(2.0 * pi)", MPINS),
    ("loss_gradient_factor", "mlp_oracle.c",
     "d[off[L] + i] = 2.0 * e * scale;", "d[off[L] + i] = e * scale;", MPINS),
    ("bias_gradient_doubled", "mlp_oracle.c",
     "gb[i] += dz[i];", "gb[i] += 2.0 * dz[i];", MPINS),
    ("adam_bias_corrections_swapped", "mlp_oracle.c",
     "p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);",
     "p[i] -= lr * (m[i] / c2) / (sqrt(v[i] / c1) + eps);", MPINS),
    # the single-box PTA loop (Sec. 3.1)
    ("load_without_the_offset", "pta.py",
     "return p.rate * (t + p.delta) * np.asarray(p.pattern, float)",
     "return p.rate * t * np.asarray(p.pattern, float)", PTAPINS),
    ("difference_quotient_reversed", "pta.py",
     "        lpdot = (sL2 / n2 - sL1 / n1) / p.delta\n        rhodot",
     "        lpdot = (sL1 / n1 - sL2 / n2) / p.delta\n        rhodot", PTAPINS),
    ("jump_restarts_from_the_first_burst", "pta.py",
     "                xyz = x2\n                jumps += 1", "                xyz = x1\n                jumps += 1", PTAPINS),
    ("extension_condition_reversed", "pta.py",
     "while np.linalg.norm(sL1 / n1) > np.linalg.norm(sL2 / n2)",
     "while np.linalg.norm(sL1 / n1) < np.linalg.norm(sL2 / n2)", PTAPINS),
    ("slow_step_from_the_earlier_average", "pta.py",
     "p.strain_step / max(np.linalg.norm(sL2 / n2), 1e-300)",
     "p.strain_step / max(np.linalg.norm(sL1 / n1), 1e-300)", PTAPINS),
    ("density_not_averaged", "pta.py",
     "RL, Rr = sL / n, sr / n", "RL, Rr = sL / n, sr", PTAPINS),
    ("microstructure_not_carried", "pta.py",
     "        xyz = x2\n        t += h", "        t += h", PTAPINS),
    # the block front end of the coupling (Sec. 4.2)
    ("block_average_by_count", "blocks.py",
     "volume += w[g]", "volume += 1.0", BLOCKPINS),
    ("extrapolation_sign", "blocks.py",
     "B = A + delta_star / dt_prev * (A - _full(T_km1[r]))",
     "B = A - delta_star / dt_prev * (A - _full(T_km1[r]))", BLOCKPINS),
    ("gap_magnification_inverted", "blocks.py",
     "mag[r] = gap_min / gap", "mag[r] = gap / gap_min", BLOCKPINS),
    ("rate_not_rescaled_back", "blocks.py",
     "lpdot[r] = (R2[r] - R1[r]) / p.delta_star / mag[r]",
     "lpdot[r] = (R2[r] - R1[r]) / p.delta_star * mag[r]", BLOCKPINS),
    ("strain_update_without_dt", "blocks.py",
     'Lp = state["Lp"] + state["Lpdot"] * dt_prev', 'Lp = state["Lp"] + state["Lpdot"]', BLOCKPINS),
    ("lock_step_checks_one_block", "blocks.py",
     "<= p.tol_rho * abs(cur_rho[r]) for r in range(R))",
     "<= p.tol_rho * abs(cur_rho[r]) for r in range(min(R, 1)))", BLOCKPINS),
]

# Runs one pin file against a copy of the oracle package: argv[1] is the
# directory that holds the copy, argv[2] the library it is to load.  The copy
# is imported before pytest starts, so every test module gets it from
# sys.modules; the package loads its library lazily, so pointing it at
# argv[2] before the first call is enough.
RUNNER = (
    "import os, sys\n"
    "sys.path.insert(0, sys.argv[1])\n"
    "import oracle\n"
    "assert os.path.dirname(os.path.dirname(oracle.__file__)) == sys.argv[1], oracle.__file__\n"
    "lib = sys.argv[2]\n"
    "oracle._LIB = lib\n"
    "oracle.build = lambda force=False: lib\n"
    "import pytest\n"
    "sys.exit(pytest.main(sys.argv[3:]))\n"
)


def _compile(pkg, out):
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", "-o", out,
           *[os.path.join(pkg, f) for f in SOURCES], "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _build_copy(workdir, mutant, real_lib):
    """Copy the oracle package into workdir/oracle and plant the mutant
    (None: none).  C sources that changed (or the unmutated copy) are
    compiled as the oracle's build does; a Python mutant loads the real
    library.  Returns (workdir, library path)."""
    pkg = os.path.join(workdir, "oracle")
    shutil.copytree(ORACLE, pkg, ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    if mutant is None:
        return workdir, _compile(pkg, os.path.join(workdir, "liboracle.so"))
    name, fname, old, new, _ = mutant
    path = os.path.join(pkg, fname)
    text = open(path).read()
    assert text.count(old) == 1, "%s: the text to mutate occurs %d times" % (name, text.count(old))
    open(path, "w").write(text.replace(old, new))
    if fname.endswith(".c"):
        return workdir, _compile(pkg, os.path.join(workdir, "liboracle.so"))
    return workdir, real_lib


def _run_pins(workdir, lib, pin_file, threads=2):
    """Exit status of the pin file against the copy (0: every pin passed)."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads),
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    args = [sys.executable, "-c", RUNNER, workdir, lib, pin_file, "-x", "-q", "-m", "not gpu",
            "-p", "no:cacheprovider"]
    if pin_file in DESELECT:
        args += ["-k", DESELECT[pin_file]]
    r = subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _workers():
    return max(1, min(8, (os.cpu_count() or 2) // 2))


@pytest.fixture(scope="module")
def real_lib():
    import oracle
    return oracle.build()


def test_unmutated_copy_passes_every_pin(tmp_path, real_lib):
    workdir, lib = _build_copy(str(tmp_path), None, real_lib)
    # the PTA pins (oracle bursts) alone on every core, then the others together
    results = [(PTAPINS, _run_pins(workdir, lib, PTAPINS, threads=os.cpu_count() or 2))]
    rest = [f for f in ALL_PINS if f != PTAPINS]
    with concurrent.futures.ThreadPoolExecutor(max_workers=_workers()) as ex:
        results += list(ex.map(lambda pins: (pins, _run_pins(workdir, lib, pins)), rest))
    for pins, (rc, out) in results:
        assert rc == 0, "the harness fails the unmutated oracle on %s:\n%s" % (pins, out)


def test_every_planted_mistake_fails_a_pin(tmp_path, real_lib):
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)

    def one(m):
        workdir, lib = _build_copy(str(tmp_path / m[0]), m, real_lib)
        return m[0], _run_pins(workdir, lib, m[4])

    # the PTA pins cost the most (oracle bursts): start them first
    order = sorted(MUTANTS, key=lambda m: m[4] != PTAPINS)
    with concurrent.futures.ThreadPoolExecutor(max_workers=_workers()) as ex:
        results = list(ex.map(one, order))
    survivors = [name for name, (rc, _) in results if rc == 0]
    assert not survivors, "planted mistakes that no pin catches: %s" % survivors
    # a pin failed (exit status 1), not the harness (collection errors, crashes)
    other = [(name, rc, out[-400:]) for name, (rc, out) in results if rc != 1]
    assert not other, "mutants that ended otherwise than by a failing pin: %s" % other
