"""The host-side parity tests of the product against planted mistakes (CPU).

The product's slow-time drivers (the single-box PTA loop of Sec. 3.1 in
`pta.py`, the block front end of Sec. 4.2 in `blocks.py`) are checked on the
CPU against the oracle's independent loops, with every burst answered by the
oracle on the host.  Here each driver gets one plausible mistake at a time
(a textual replacement that matches exactly once, in a copy of the module
that the subprocess loads in place of the real one), and those parity tests
must fail; the unmodified copy, loaded the same way, must pass them.
The kernels' own parity tests need a GPU and are not covered here.
"""

import concurrent.futures
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2005_02498_gb300")

PTA_TESTS = ["tests/test_pta_oracle.py", "-k", "product_pta_driver"]
BLOCK_TESTS = ["tests/test_blocks.py", "-k", "block_driver or stress_step_control or synthetic_coupling"]

# (name, module, text, replacement)
MUTANTS = [
    ("jump_keeps_the_first_state", "pta",
     "state, jumps = s2, jumps + 1", "state, jumps = s1, jumps + 1"),
    ("microstructure_not_carried", "pta",
     "        state = s2\n        t += h", "        t += h"),
    ("extension_from_the_second_state", "pta",
     "ctx.set_state(s1)\n            ctx.set_applied_stress(load(t - p.delta))",
     "ctx.set_state(s2)\n            ctx.set_applied_stress(load(t - p.delta))"),
    ("load_without_the_offset", "pta",
     "load = lambda t: p.rate * (t + p.delta) * pattern", "load = lambda t: p.rate * t * pattern"),
    ("slow_step_from_the_earlier_average", "pta",
     "p.strain_step / max(np.linalg.norm(a2.lp), 1e-300)", "p.strain_step / max(np.linalg.norm(a1.lp), 1e-300)"),
    ("density_criterion_dropped", "pta",
     "dr = abs(cur[1] - prev[1]) <= p.tol_rho * abs(cur[1])", "dr = True"),
    ("density_rate_halved", "pta",
     "rhodot = (a2.rho - a1.rho) / p.delta", "rhodot = (a2.rho - a1.rho) / p.delta / 2"),
    ("rate_not_rescaled_back", "blocks",
     "lpdot = (R2 - R1) / p.delta_star / mag[:, None, None]", "lpdot = (R2 - R1) / p.delta_star * mag[:, None, None]"),
    ("strain_update_with_delta_star", "blocks",
     "self.Lp = self.Lp + self.Lpdot * dt_prev", "self.Lp = self.Lp + self.Lpdot * p.delta_star"),
    ("lock_step_stops_at_the_first_block", "blocks",
     "if np.all(ok_lp & ok_rho):", "if np.any(ok_lp & ok_rho):"),
    ("step_quartered", "blocks",
     "dt = max(0.5 * dt, p.delta_star)", "dt = max(0.25 * dt, p.delta_star)"),
    ("density_rate_not_rescaled", "blocks",
     "rhodot = (rho2 - rho1) / p.delta_star / mag", "rhodot = (rho2 - rho1) / p.delta_star"),
]

# Loads argv[2] as the package's module argv[1] before pytest starts, so the
# tests import the copy.
RUNNER = (
    "import importlib.util, sys\n"
    "import paper_2005_02498_gb300 as pkg\n"
    "name, path = sys.argv[1], sys.argv[2]\n"
    "spec = importlib.util.spec_from_file_location('paper_2005_02498_gb300.' + name, path)\n"
    "mod = importlib.util.module_from_spec(spec)\n"
    "sys.modules[spec.name] = mod\n"
    "spec.loader.exec_module(mod)\n"
    "setattr(pkg, name, mod)\n"
    "import pytest\n"
    "sys.exit(pytest.main(sys.argv[3:]))\n"
)


def _copy(workdir, module, mutant):
    os.makedirs(workdir, exist_ok=True)
    text = open(os.path.join(PKG, module + ".py")).read()
    if mutant is not None:
        name, _, old, new = mutant
        assert text.count(old) == 1, "%s: the text to mutate occurs %d times" % (name, text.count(old))
        text = text.replace(old, new)
    path = os.path.join(workdir, module + ".py")
    open(path, "w").write(text)
    return path


def _run(module, path, threads=2):
    tests = PTA_TESTS if module == "pta" else BLOCK_TESTS
    env = dict(os.environ, OMP_NUM_THREADS=str(threads),
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    args = [sys.executable, "-c", RUNNER, module, path, *tests, "-x", "-q", "-m", "not gpu",
            "-p", "no:cacheprovider"]
    r = subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _workers():
    return max(1, min(8, (os.cpu_count() or 2) // 2))


def test_unmodified_copies_pass_the_parity_tests(tmp_path):
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        results = list(ex.map(lambda m: (m, _run(m, _copy(str(tmp_path / m), m, None),
                                                 threads=max(2, (os.cpu_count() or 2) // 2))), ("pta", "blocks")))
    for module, (rc, out) in results:
        assert rc == 0, "the harness fails the unmodified %s:\n%s" % (module, out)


def test_every_planted_mistake_fails_a_parity_test(tmp_path):
    names = [m[0] + m[1] for m in MUTANTS]
    assert len(set(names)) == len(names)

    def one(m):
        return m[0], _run(m[1], _copy(str(tmp_path / (m[1] + "_" + m[0])), m[1], m))

    with concurrent.futures.ThreadPoolExecutor(max_workers=_workers()) as ex:
        results = list(ex.map(one, sorted(MUTANTS, key=lambda m: m[1] != "pta")))
    survivors = [name for name, (rc, _) in results if rc == 0]
    assert not survivors, "planted mistakes that no parity test catches: %s" % survivors
    other = [(name, rc, out[-400:]) for name, (rc, out) in results if rc != 1]
    assert not other, "mutants that ended otherwise than by a failing test: %s" % other
