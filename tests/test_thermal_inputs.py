"""The stored thermally unfolded chains (X_N run 2 ns at 600 K by the FP64 oracle, written
by oracle/unfold.py) load with their recorded hash and are unfolded, intact chains."""
import os

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n_res", [19, 35, 75])
def test_stored_unfolded_chain(n_res):
    if synth.chain.thermal_unfolded(n_res) is None:
        pytest.skip("no stored unfolded chain of this size")
    c = synth.make_chain(n_res, seed=1)
    x = c.x_unfolded
    assert x.shape == c.x_native.shape and np.all(np.isfinite(x))
    assert not np.array_equal(x, c.x_coil)
    # bonds stay near their rest lengths (a few thermal widths at 600 K)
    b = np.array(c.bonds)
    r = np.linalg.norm(x[b[:, 1]] - x[b[:, 0]], axis=1)
    assert np.all(np.abs(r - np.asarray(c.b0)) < 0.03)
    # fewer native contacts formed than in X_N: z of Eq. (zrMD) measured from X_N grows
    q = lambda y: sum(oracle.contact_C(np.linalg.norm(y[j] - y[i])) for i, j in c.contacts)
    assert q(x) < 0.6 * q(c.x_native)


def test_stored_file_hash_is_checked(tmp_path, monkeypatch):
    src = synth.chain.thermal_unfolded(19)
    if src is None:
        pytest.skip("no stored unfolded chain")
    with open(os.path.join(synth.chain._THERMAL_DIR, "chain_r19_s1_600K_2ns.txt")) as f:
        lines = f.readlines()
    lines[1] = lines[1].replace(lines[1].split()[0], "%.17g" % (float(lines[1].split()[0]) + 1e-9), 1)
    (tmp_path / "chain_r19_s1_600K_2ns.txt").write_text("".join(lines))
    monkeypatch.setattr(synth.chain, "_THERMAL_DIR", str(tmp_path))
    with pytest.raises(ValueError):
        synth.chain.thermal_unfolded(19)
