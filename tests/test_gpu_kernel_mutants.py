"""The GPU parity tests against mistakes planted in the kernels (opt-in).

Each mutant is a copy of the package whose CUDA sources carry one plausible
mistake (a textual replacement that matches exactly once): a dropped or
sign-flipped coefficient term, a wrong Kahan compensation, swapped shape
function weights, a neighbour index swapped for the other neighbour, the
Euler step's sign, a wrong mass-matrix entry.  Every planted mistake is
arithmetic or replaces an index by another valid one, so no mutant can
access memory outside its buffers or change a wait.  The translation units
that include the mutated file are recompiled into the copy, linked with
the library's other objects, and the parity tests against the oracle for
that part of the path run on the copy in a subprocess; they must fail.  The
unmodified copy, built the same way, must pass them.

Opt-in: it needs a GPU, nvcc and several minutes, so it runs only with
PTADD_KERNEL_MUTANTS=1, e.g.
    PTADD_KERNEL_MUTANTS=1 python -m pytest tests/test_gpu_kernel_mutants.py -m kernel_mutants -q
and is selected neither by -m gpu nor by -m "not gpu".
"""

import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2005_02498_gb300")

pytestmark = [
    pytest.mark.kernel_mutants,
    pytest.mark.skipif(os.environ.get("PTADD_KERNEL_MUTANTS") != "1",
                       reason="opt-in: set PTADD_KERNEL_MUTANTS=1 on a machine with a GB300"),
]

FP64 = ["tests/test_gpu_parity.py", "-k", "nodal_forces_match_oracle or burst_small_loops_100 or zero_length"]
MIXED = ["tests/test_gpu_mixed.py", "-k", "mixed_forces_match_oracle or large_workload_sampled or rates_small"]
CONSISTENT = ["tests/test_gpu_consistent_mobility.py", "-k", "burst_matches_oracle"]

# (name, file under csrc/, text, replacement, parity tests)
MUTANTS = [
    # the FP64 field formula (Sec. 2.1)
    ("fp64_b_term_sign", "seg_field.cuh", "sb = fma(qR, B0, sb);", "sb = fma(-qR, B0, sb);", FP64),
    ("fp64_kn_dropped", "seg_field.cuh",
     "const double C1 = fma(nra2, K3, kn * J1);", "const double C1 = fma(nra2, K3, J1);", FP64),
    ("fp64_one_side_Aw_sign", "seg_field.cuh",
     "const double Z = fma(isum, fma(-d2, i12, ssum), T * ssum);",
     "const double Z = fma(isum, fma(d2, i12, ssum), T * ssum);", FP64),
    ("fp64_straddling_J0_sign", "seg_field.cuh",
     "J0 = same ? (Li * rden) * one_pm : (p - m) * rden;", "J0 = same ? (Li * rden) * one_pm : (p + m) * rden;", FP64),
    # the packed FP32 formula and its sums
    ("mixed_cb_from_A0", "pair_tile.cuh", "C.cb = mul2(qR, B0);", "C.cb = mul2(qR, A0);", MIXED),
    ("mixed_Aw_sign", "pair_tile.cuh",
     "const float2 Aw = fma2(neg2(d2), i12, ssum);", "const float2 Aw = fma2(d2, i12, ssum);", MIXED),
    ("mixed_kahan_compensation_sign", "pair_tile.cuh", "c = sub2(sub2(t, s), y);", "c = sub2(sub2(s, t), y);", MIXED),
    ("mixed_b_term_not_closed", "pair_tile.cuh",
     "for (int e = 0; e < 3; ++e) SG[p][e] = fma2(SB[p], bt2[e], SG[p][e]);",
     "for (int e = 0; e < 3; ++e) SG[p][e] = add2(SG[p][e], f2(0.0f));", MIXED),
    ("mixed_b_term_without_Q", "pair_tile.cuh",
     "SB[p] = fma2(C[p].Q, C[p].cb, SB[p]);", "SB[p] = add2(C[p].cb, SB[p]);", MIXED),
    # the shared epilogue: shape functions and the applied stress
    ("shape_function_weights_swapped", "pair_tile.cuh",
     "const double we = gl4_w(qp) * gl4_xi(qp), ws = gl4_w(qp) - we;",
     "const double ws = gl4_w(qp) * gl4_xi(qp), we = gl4_w(qp) - ws;", FP64),
    ("applied_stress_times_b_index", "pair_tile.cuh",
     "const double sb0 = s[0] * bt[0] + s[5] * bt[1] + s[4] * bt[2];",
     "const double sb0 = s[0] * bt[0] + s[4] * bt[1] + s[5] * bt[2];", FP64),
    # the node and step kernels (Eq. 2.1, the Euler step)
    ("nodal_assembly_other_neighbour", "dd_kernels.cu",
     "F[0] += fp[0 * n + a] + fp[3 * n + p];", "F[0] += fp[0 * n + a] + fp[3 * n + nx];", FP64),
    ("euler_step_sign", "dd_kernels.cu",
     "const double nxp = __dadd_rn(pos[i], __dmul_rn(vel[i], dt));",
     "const double nxp = __dsub_rn(pos[i], __dmul_rn(vel[i], dt));", FP64),
    ("consistent_mass_off_diagonal", "dd_kernels.cu",
     "const double ct = last ? 0.0 : Lt / 6.0;", "const double ct = last ? 0.0 : Lt / 3.0;", CONSISTENT),
]

# translation units that include each header
INCLUDERS = {"seg_field.cuh": ["dd_kernels.cu", "batch.cu"], "pair_tile.cuh": ["dd_kernels.cu", "batch.cu"]}

# Runs the parity tests against the copy held in argv[1]: it is imported
# before pytest starts, so every test gets it from sys.modules, and its
# library is the one under its own _lib.
RUNNER = (
    "import os, sys\n"
    "sys.path.insert(0, sys.argv[1])\n"
    "import paper_2005_02498_gb300 as P\n"
    "assert os.path.dirname(os.path.dirname(os.path.abspath(P.__file__))) == sys.argv[1], P.__file__\n"
    "import pytest\n"
    "sys.exit(pytest.main(sys.argv[2:]))\n"
)


def _make_copy(workdir, mutant):
    """Copy the package (with its built objects) and the header into
    workdir, plant the mutant (None: none), recompile the translation units
    that see the mutated file and relink the copy's library."""
    from paper_2005_02498_gb300 import build as B
    dst = os.path.join(workdir, "paper_2005_02498_gb300")
    shutil.copytree(PKG, dst, ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "include"), os.path.join(workdir, "include"))
    units = []
    if mutant is not None:
        name, fname, old, new, _ = mutant
        path = os.path.join(dst, "csrc", fname)
        text = open(path).read()
        assert text.count(old) == 1, "%s: the text to mutate occurs %d times" % (name, text.count(old))
        open(path, "w").write(text.replace(old, new))
        units = INCLUDERS.get(fname, [fname])
    objdir = os.path.join(dst, "_lib", "obj")
    for u in units:
        cmd = [B.nvcc(), *B.ARCH, *B.NVCC_FLAGS, "-c", os.path.join(dst, "csrc", u), "-o", os.path.join(objdir, u + ".o")]
        subprocess.run(cmd, check=True, capture_output=True)
    lib = os.path.join(dst, "_lib", "libptadd.so")
    objs = sorted(os.path.join(objdir, f) for f in os.listdir(objdir) if f.endswith(".o"))
    subprocess.run([B.nvcc(), *B.ARCH, "-shared", "-o", lib, *objs, "-cudart", "static"], check=True,
                   capture_output=True)
    return workdir


def _run(workdir, tests):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    args = [sys.executable, "-c", RUNNER, workdir, *tests, "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider"]
    r = subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def built():
    from paper_2005_02498_gb300 import build as B
    return B.build()  # the library and the objects the copies start from


def test_unmodified_copy_passes_the_parity_tests(tmp_path, built):
    workdir = _make_copy(str(tmp_path), None)
    for tests in (FP64, MIXED, CONSISTENT):
        rc, out = _run(workdir, tests)
        assert rc == 0, "the harness fails the unmodified kernels on %s:\n%s" % (tests[0], out)


def test_every_kernel_mistake_fails_a_parity_test(tmp_path, built):
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    # the builds in parallel (host work), the GPU runs one at a time
    with concurrent.futures.ThreadPoolExecutor(max_workers=4) as ex:
        dirs = list(ex.map(lambda m: _make_copy(str(tmp_path / m[0]), m), MUTANTS))
    results = [(m[0], _run(d, m[4])) for m, d in zip(MUTANTS, dirs)]
    survivors = [name for name, (rc, _) in results if rc == 0]
    assert not survivors, "kernel mistakes that no parity test catches: %s" % survivors
    other = [(name, rc, out[-400:]) for name, (rc, out) in results if rc != 1]
    assert not other, "mutants that ended otherwise than by a failing test: %s" % other
