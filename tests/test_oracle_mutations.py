"""The oracle's pins catch plausible mistakes in the oracle.

Each case plants one mistake in a scratch copy of oracle/: a wrong neighbour,
a flipped sign, a dropped conjugate, a wrong power of the scale factor, a
wrong constant.  It then runs the pin files that cover that part in a
subprocess and requires at least one pin to fail: a real test failure, not a
build or collection error.  An unmutated copy must pass the same files, so a
failure is the mistake's doing.

The cases cover the scalar sector (section 4: the Laplacian of the kernel,
the section-8.1 potential, the Hamiltonian energies and the scale-factor
kernel of section 4.3.2), the compact U(1) sector (section 5.3: the magnetic
force, the current, the parallel transport), the SU(2) toolkit (section
3.2.3: quaternion conjugate and product), the spectra and the vacuum initial
conditions of section 3.1, the counter-based generator, the surrogate MLP's
activation derivative and the equation of state.

Only oracle/ is touched, and only in a temporary directory; no GPU is used.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, oracle file, original text, planted text, pin files)
CASES = [
    ("laplacian-wrong-neighbour", "lattice_oracle.c",
     "f[site(N, x, y, wrap(z + 1, N))] + f[site(N, x, y, wrap(z - 1, N))] -",
     "f[site(N, x, y, wrap(z + 1, N))] + f[site(N, x, y, wrap(z + 1, N))] -", ["test_oracle_scalar.py"]),
    ("laplacian-diagonal", "lattice_oracle.c", "6.0 * f[n]) * idx2;", "4.0 * f[n]) * idx2;",
     ["test_oracle_scalar.py"]),
    ("interaction-force-sign", "lattice_oracle.c", "*dchi = m->q * phi * phi * chi;",
     "*dchi = -m->q * phi * phi * chi;", ["test_oracle_scalar.py"]),
    ("interaction-energy-factor", "lattice_oracle.c", "? 0.5 * m->q * phi * phi * chi * chi : 0.0;",
     "? m->q * phi * phi * chi * chi : 0.0;", ["test_oracle_scalar.py"]),
    ("kinetic-energy-a-power", "lattice_oracle.c", "out[i] = sk[i] / V / (2.0 * a6);",
     "out[i] = sk[i] / V / (2.0 * a2);", ["test_oracle_scalar.py"]),
    ("friedmann-kernel-coefficient", "lattice_oracle.c", "           ((m->alpha - 2.0) * EK + m->alpha * EG",
     "           ((m->alpha - 1.0) * EK + m->alpha * EG", ["test_oracle_scalar.py"]),
    ("kernel-gradient-a-power", "lattice_oracle.c",
     "const double a1 = pow(a, 1.0 + m->alpha), a3 = pow(a, 3.0 + m->alpha);\n",
     "const double a1 = pow(a, 2.0 + m->alpha), a3 = pow(a, 3.0 + m->alpha);\n", ["test_oracle_scalar.py"]),
    ("drift-a-power", "lattice_oracle.c", "drift(m, phi, pi, h * pow(ah, -(3.0 - m->alpha)));",
     "drift(m, phi, pi, h * pow(ah, -(1.0 - m->alpha)));", ["test_oracle_scalar.py"]),
    ("scale-factor-half-step", "lattice_oracle.c",
     "        *a = ah + 0.5 * h * bh;\n        kick(m, phi, pi, *a, 0.5 * h, K);\n        orc_scalar_energies(",
     "        *a = ah + h * bh;\n        kick(m, phi, pi, *a, 0.5 * h, K);\n        orc_scalar_energies(",
     ["test_oracle_scalar.py"]),
    ("u1-magnetic-force-sign", "lattice_oracle.c", "return m->noncompact ? t : sin(t); }",
     "return m->noncompact ? t : -sin(t); }", ["test_oracle_u1.py"]),
    ("u1-current-sign", "lattice_oracle.c", "const double cur = pr[n] * ui - pim[n] * ur;",
     "const double cur = pim[n] * ur - pr[n] * ui;", ["test_oracle_u1.py"]),
    ("u1-backward-link-conjugate", "lattice_oracle.c", "const double wr = cos(tm) * pr[nm] - sin(tm) * pim[nm];",
     "const double wr = cos(tm) * pr[nm] + sin(tm) * pim[nm];", ["test_oracle_u1.py"]),
    ("su2-quaternion-conjugate", "lattice_oracle.c", "r[0] = q[0]; r[1] = -q[1]; r[2] = -q[2]; r[3] = -q[3];",
     "r[0] = q[0]; r[1] = q[1]; r[2] = -q[2]; r[3] = -q[3];", ["test_oracle_su2.py"]),
    ("su2-product-cross-term", "lattice_oracle.c",
     "const double r1 = p[0] * q[1] + q[0] * p[1] - (p[2] * q[3] - p[3] * q[2]);",
     "const double r1 = p[0] * q[1] + q[0] * p[1] + (p[2] * q[3] - p[3] * q[2]);", ["test_oracle_su2.py"]),
    ("spectrum-power-of-k", "spectra.py", "Delta = k ** 3 / (2 * np.pi ** 2)", "Delta = k ** 2 / (2 * np.pi ** 2)",
     ["test_oracle_ic.py", "test_oracle_observe.py"]),
    ("ic-self-conjugate-amplitude", "ic.py", "F = np.where(selfc, np.sqrt(2.0) * G.real + 0j, F)",
     "F = np.where(selfc, G.real + 0j, F)", ["test_oracle_ic.py"]),
    ("philox-weyl-constant", "philox.py", "\nW0 = 0x9E3779B9\n", "\nW0 = 0x9E3779B8\n", ["test_oracle_ic.py"]),
    ("gelu-derivative", "mlp.py", "x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)",
     "x * np.exp(-x * x) / np.sqrt(2.0 * np.pi)", ["test_oracle_mlp.py"]),
    ("w-pressure", "observe.py", "out[1] = (EK - EG / 3.0 - EV) / rho", "out[1] = (EK - EG - EV) / rho",
     ["test_oracle_observe.py"]),
]

PIN_FILES = sorted({p for case in CASES for p in case[4]})


def _scratch_copy(dst):
    """oracle/ and the CPU pin files (with what they import) under dst."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ["__init__.py", "conftest.py", "inputs.py"] + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))


def _run_pins(dst, pins):
    env = dict(os.environ, PYTHONPATH=dst, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       ["tests/" + p for p in pins], cwd=dst, env=env, capture_output=True, text=True,
                       timeout=600)
    lines = r.stdout.strip().splitlines()
    return r.returncode, (lines[-1] if lines else r.stderr[-400:])


def _one(tmp, case):
    name, fname, old, new, pins = case
    dst = os.path.join(tmp, name)
    _scratch_copy(dst)
    path = os.path.join(dst, "oracle", fname)
    with open(path) as fh:
        src = fh.read()
    if src.count(old) != 1:
        return name, (None, "the original text occurs %d times in %s" % (src.count(old), fname))
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    # the mutant must still build, so that a pin fails on its arithmetic, not on gcc
    b = subprocess.run([sys.executable, "-c", "from oracle import build; build.build(force=True)"], cwd=dst,
                       env=dict(os.environ, PYTHONPATH=dst), capture_output=True, text=True, timeout=300)
    if b.returncode != 0:
        return name, (None, "the mutant does not build: " + b.stderr[-300:])
    return name, _run_pins(dst, pins)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Run the unmutated copy and every mutant, four at a time."""
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    base = os.path.join(tmp, "unmutated")
    _scratch_copy(base)
    clean = _run_pins(base, PIN_FILES)
    with ThreadPoolExecutor(max_workers=4) as pool:
        res = dict(pool.map(lambda c: _one(tmp, c), CASES))
    return clean, res


def test_unmutated_copy_passes_the_pins(outcomes):
    rc, summary = outcomes[0]
    assert rc == 0 and "passed" in summary and "failed" not in summary, summary


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(outcomes, name):
    clean_rc, _ = outcomes[0]
    assert clean_rc == 0
    rc, summary = outcomes[1][name]
    assert rc is not None, summary
    # exit status 1 with "failed" and no "error": a pin failed, the copy built and collected
    assert rc == 1 and "failed" in summary and "error" not in summary, summary
