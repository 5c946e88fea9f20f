"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake -- a dropped term, a wrong sign, index or
operand, a transposed matrix, a wrong constant -- in a temporary copy of
oracle/ and runs tests/test_oracle_pins.py against that copy in a child
process; the pins must fail.  The real oracle is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

E, S = "oracle/energies.py", "oracle/solver.py"
MUTATIONS = [
    # image warping (Fig. 24)
    (E, "Rv = np.stack([c * v[0] - s * v[1], s * v[0] + c * v[1]])",
        "Rv = np.stack([c * v[0] + s * v[1], -s * v[0] + c * v[1]])"),            # clockwise rotation
    (E, "valid = inb & ~mask & ~mask[nyc, nxc]", "valid = inb & ~mask"),          # masked neighbour kept
    (E, "vals += [-sw * (-s * v[0] - c * v[1]), -sw * (c * v[0] - s * v[1])]",
        "vals += [sw * (-s * v[0] - c * v[1]), -sw * (c * v[0] - s * v[1])]"),    # sign of dr/dtheta
    (E, "rows += [rr, rr[jf]]", "rows += [rr, rr]"),                                # wrong row of the far end
    (E, "js.append((np.clip(ny, 0, H - 1) * W + np.clip(nx, 0, W - 1))[valid])",
        "js.append((np.clip(nx, 0, H - 1) * W + np.clip(ny, 0, W - 1))[valid])"),  # x / y swapped
    # ARAP mesh (Fig. 25)
    (E, "    R = Rz @ Ry @ Rx", "    R = Rx @ Ry @ Rz"),                            # Euler order
    (E, "cols += [i * V + a, i * V + b]", "cols += [i * V + a, i * V + a]"),       # far-end column
    (E, "cols.append((3 + mm) * V + a)", "cols.append((3 + mm) * V + b)"),         # rotation of the wrong end
    (E, "reg = self.s_w * ((O[:, a] - O[:, b]) - Rv)", "reg = self.s_w * ((O[:, a] - O[:, b]) + Rv)"),
    (E, "fit = self.s_f * (O[:, self.h] - self.C)", "fit = self.prob.w_fit * (O[:, self.h] - self.C)"),  # weight not rooted
    # warp on a graph (Fig. 18)
    (E, "dRv = np.stack([-s * v[0] - c * v[1], c * v[0] - s * v[1]])",
        "dRv = np.stack([-s * v[0] + c * v[1], c * v[0] - s * v[1]])"),
    # volumetric ARAP (Fig. 31)
    (E, "vals.append(-sw * np.einsum('ej,ej->e', dR[mm][:, i, :], v))",
        "vals.append(-sw * np.einsum('ej,ej->e', dR[mm][:, :, i], v))"),           # transposed derivative
    (E, "                    src[axis], dst[axis] = slice(1, None), slice(0, -1)",
        "                    src[axis], dst[axis] = slice(0, -1), slice(1, None)"),  # one direction only
    # embedded deformation (Fig. 28)
    (E, "col = [Rm[:, k, :] for k in range(3)]", "col = [Rm[k, :, :] for k in range(3)]"),   # rows, not columns
    (E, "np.sum(col[i] * col[j], axis=0) - (1.0 if i == j else 0.0)", "np.sum(col[i] * col[j], axis=0)"),
    (E, "vals.append(2.0 * sr * Rm[r, i])", "vals.append(sr * Rm[r, i])"),           # factor 2 dropped
    (E, "                vals.append(-sw * v[c])", "                vals.append(sw * v[c])"),
    (E, "Rv = np.einsum('rce,ce->re', Rm[:, :, a], v)", "Rv = np.einsum('rce,re->ce', Rm[:, :, a], v)"),
    # PCG / GN / LM (Sec. 4)
    (S, "        beta = float(rd(rho_new / rho))", "        beta = float(rd(rho / rho_new))"),
    (S, "        z = rd(Minv * r)", "        z = rd(r)"),
    (S, "        x = rd(x + d)", "        x = rd(x - d)"),
    (S, "lam = lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)",
        "lam = lam * min(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)"),
    (S, "        r = rd(r - alpha * q)", "        r = rd(r - alpha * p)"),
    (S, "pred = E - float(Fl @ Fl)", "pred = E + float(Fl @ Fl)"),
    (S, "        q = q + lam * Dc * p", "        q = q + lam * p"),
]


def run_pins_on_copy(tmp_path, path=None, pattern=None, replacement=None):
    """Copies the oracle (with one mistake planted, if given), its pins and
    their fixtures to tmp_path and runs the pins there; returns the result."""
    work = tmp_path / "mut"
    work.mkdir()
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "paper_1604_06525_gb300"), work / "paper_1604_06525_gb300",
                    ignore=shutil.ignore_patterns("__pycache__", "_lib", "_build", "*.so"))
    (work / "tests").mkdir()
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), work / "tests" / "golden")
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), work / "tests" / f)
    if path is not None:
        target = work / path
        src = target.read_text()
        assert src.count(pattern) >= 1, f"pattern not found in {path}: {pattern}"
        target.write_text(src.replace(pattern, replacement, 1))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                           "-p", "no:cacheprovider", "-m", "not gpu"],
                          cwd=work, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes(tmp_path):
    """Control: the harness itself works -- the copied oracle passes its pins."""
    res = run_pins_on_copy(tmp_path)
    assert res.returncode == 0, res.stdout[-2000:]
    assert " passed" in res.stdout


@pytest.mark.parametrize("path,pattern,replacement", MUTATIONS,
                         ids=[f"{i:02d}" for i in range(len(MUTATIONS))])
def test_pins_catch_planted_mistake(tmp_path, path, pattern, replacement):
    res = run_pins_on_copy(tmp_path, path, pattern, replacement)
    assert res.returncode == 1, f"mutation not caught: {pattern!r} -> {replacement!r}\n{res.stdout[-2000:]}"
    assert " failed" in res.stdout, res.stdout[-2000:]
