"""The oracle's pins against planted mistakes: each case copies the oracle into a scratch directory, plants one
plausible mistake (a dropped factor, a wrong sign, a transposed or mis-indexed operand) and runs the pin tests of that
module there; the pins must fail. This checks the pins, not the oracle: the oracle in the repository is untouched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle file, text, planted replacement, pin test files that must catch it, what the mistake is)
CASES = [
    ("soap.py", 'pair_species = a_all[nl["nbr_j"]]', "pair_species = a_all[centres[pair_centre]]",
     ["test_oracle_soap.py"], "neighbour j's term in the centre's species block (species channel of c)"),
    ("soap.py", "k = 1.0 / sqrt(2 * l + 1) if h.ps_norm else 1.0\n        full[:, l]",
     "k = 1.0 / (2 * l + 1) if h.ps_norm else 1.0\n        full[:, l]",
     ["test_oracle_soap.py"], "power-spectrum normalisation (2l+1)^-1 instead of (2l+1)^-1/2"),
    ("soap.py", "W + np.transpose(W, (0, 2, 1))", "W", ["test_oracle_soap.py"],
     "adjoint without the transposed half of the packed weights"),
    ("soap.py", 's1 = np.einsum("pnk,pnk,pk->p", ch, dR, Y)', 's1 = np.einsum("pnk,pnk,pk->p", ch, R, Y)',
     ["test_oracle_soap.py"], "radial derivative replaced by the radial value in the pair gradient"),
    ("ylm.py", "Y[:, lm_index(l, -m)] = f * P[l, m] * S[m]", "Y[:, lm_index(l, -m)] = -f * P[l, m] * S[m]",
     ["test_oracle_ylm.py", "test_oracle_soap.py"], "sign of the sine harmonics"),
    ("gto.py", "return (V * (1.0 / np.sqrt(w))[None, :]) @ V.T", "return (V * (1.0 / w)[None, :]) @ V.T",
     ["test_oracle_radial.py"], "S^-1 instead of S^-1/2 in the orthonormalisation"),
    ("neighbours.py", "mask = d2 < rc2", "mask = d2 <= rc2", ["test_oracle_neighbours.py"],
     "pairs at exactly r_cut kept"),
    ("mlp.py", "vh = v / (1 - beta2 ** t)", "vh = v / (1 - beta2)", ["test_oracle_mlp.py"],
     "Adam second-moment bias correction frozen at step 1"),
    ("lambda_soap.py", "s += (-1) ** k / den", "s += 1.0 / den", ["test_oracle_lambda_soap.py"],
     "alternating sign dropped from Racah's sum"),
]


@pytest.mark.parametrize("case", CASES, ids=[c[4] for c in CASES])
def test_planted_mistake_fails_a_pin(case, tmp_path):
    fname, old, new, pins, _ = case
    for sub in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub, ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path)
    path = tmp_path / "oracle" / fname
    src = path.read_text()
    assert src.count(old) == 1, f"the text to plant into is not unique in oracle/{fname}"
    path.write_text(src.replace(old, new))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu", *[f"tests/{p}" for p in pins]],
                         cwd=tmp_path, capture_output=True, text=True, timeout=600,
                         env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert res.returncode == 1, res.stdout[-2000:] + res.stderr[-2000:]
    assert " failed" in res.stdout
