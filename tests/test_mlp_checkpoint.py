"""Checkpoint of the warm-start network (wl_mlp_save / wl_mlp_load): host code
only, no GPU. A saved parameter vector loads back bit for bit; a file with
another length, magic or shape is rejected (WL_ERR_INVALID_ARG), one whose
parameters do not match their stored hash too (WL_ERR_NONFINITE)."""
import numpy as np
import pytest

from paper_2601_11338_gb300 import wl


def params(seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(wl.wl_mlp_param_count()).astype(np.float32)
    p[:3] = [np.float32(-0.0), np.float32(1e-30), np.float32(3.4e38)]
    return p


def test_round_trip_is_bit_exact(tmp_path):
    p = params(1)
    f = tmp_path / "net.wlmlp"
    assert wl.wl_mlp_save(str(f), p) == wl.WL_OK
    q = wl.wl_mlp_load(str(f))
    assert np.array_equal(p.view(np.uint32), q.view(np.uint32))
    raw = f.read_bytes()
    assert raw[:8] == b"WLMLP001" and len(raw) == 32 + 4 * p.size
    assert int.from_bytes(raw[20:24], "little") == p.size


@pytest.mark.parametrize("damage,status", [("flip", wl.WL_ERR_NONFINITE), ("truncate", wl.WL_ERR_INVALID_ARG),
                                           ("extend", wl.WL_ERR_INVALID_ARG), ("magic", wl.WL_ERR_INVALID_ARG),
                                           ("width", wl.WL_ERR_INVALID_ARG)])
def test_damaged_files_are_rejected(tmp_path, damage, status):
    p = params(2)
    f = tmp_path / "net.wlmlp"
    wl.wl_mlp_save(str(f), p)
    raw = bytearray(f.read_bytes())
    if damage == "flip":
        raw[32 + 4 * 100] ^= 0x01
    elif damage == "truncate":
        raw = raw[:-4]
    elif damage == "extend":
        raw += b"\\0"
    elif damage == "magic":
        raw[7:8] = b"9"
    else:
        raw[12:16] = (32).to_bytes(4, "little")
    f.write_bytes(bytes(raw))
    assert wl.wl_mlp_load(str(f), allow=(status,)) is None
    with pytest.raises(wl.WLError):
        wl.wl_mlp_load(str(f))


def test_missing_file_is_rejected(tmp_path):
    assert wl.wl_mlp_load(str(tmp_path / "absent"), allow=(wl.WL_ERR_INVALID_ARG,)) is None
