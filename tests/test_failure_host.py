"""Failure detection on the host (no GPU): damaged or mismatched weight files of the learned warm
start are rejected with a clear ValueError before the library is called."""
import os

import numpy as np
import pytest

from paper_1909_13585_gb300 import learned


def test_committed_weights_pass_the_checks():
    z = learned.read_weights(learned.WEIGHTS)
    assert z["params"].size == z["adam_m"].size == z["adam_v"].size > 0


def test_truncated_file_is_rejected(tmp_path):
    raw = open(learned.WEIGHTS, "rb").read()
    bad = tmp_path / "truncated.npz"
    bad.write_bytes(raw[: len(raw) // 2])
    with pytest.raises(ValueError, match="not a readable"):
        learned.read_weights(str(bad))
    junk = tmp_path / "junk.npz"
    junk.write_bytes(os.urandom(4096))
    with pytest.raises(ValueError, match="not a readable"):
        learned.read_weights(str(junk))


def _write(tmp_path, **over):
    z = dict(learned.read_weights(learned.WEIGHTS))
    z.update(over)
    z = {k: v for k, v in z.items() if v is not None}
    path = str(tmp_path / "w.npz")
    np.savez(path, **z)
    return path


def test_missing_keys_wrong_types_and_mismatched_moments_are_rejected(tmp_path):
    with pytest.raises(ValueError, match="lacks params"):
        learned.read_weights(_write(tmp_path, params=None))
    p = learned.read_weights(learned.WEIGHTS)["params"]
    with pytest.raises(ValueError, match="float32"):
        learned.read_weights(_write(tmp_path, params=p.astype(np.float64)))
    with pytest.raises(ValueError, match="adam_m"):
        learned.read_weights(_write(tmp_path, adam_m=np.zeros(p.size - 1, np.float32)))
    q = p.copy()
    q[3] = np.nan
    with pytest.raises(ValueError, match="non-finite"):
        learned.read_weights(_write(tmp_path, params=q))
