"""The learned preconditioner's checkpoint format, read on the host (CPU only): a file written
here by the documented layout parses; foreign or corrupt headers are argument errors."""
import struct

import numpy as np
import pytest


def _lib():
    from tests.gpu_util import lib
    return lib()


def _write(path, magic=b"FELPC001", din=27, width=64, nparam=None, steps=123):
    nparam = 2 * din * width + width * width + din * din if nparam is None else nparam
    with open(path, "wb") as f:
        f.write(magic + struct.pack("<iiqii", din, width, nparam, steps, 0))
        for _ in range(3):
            f.write(np.zeros(max(nparam, 0), dtype="<f4").tobytes())
    return nparam


def test_header_roundtrip(tmp_path):
    fe = _lib()
    p = tmp_path / "lpc.bin"
    n = _write(p)
    assert fe.fe_lpc_checkpoint_info(str(p)) == (27, 64, n, 123)


@pytest.mark.parametrize("kw", [dict(magic=b"NOTLPC01"), dict(din=0), dict(nparam=0),
                                dict(steps=-1)])
def test_bad_headers_are_argument_errors(tmp_path, kw):
    fe = _lib()
    p = tmp_path / "bad.bin"
    _write(p, **kw)
    with pytest.raises(fe.FEError) as e:
        fe.fe_lpc_checkpoint_info(str(p))
    assert e.value.status == fe.FE_ERR_ARG


def test_missing_file(tmp_path):
    fe = _lib()
    with pytest.raises(fe.FEError):
        fe.fe_lpc_checkpoint_info(str(tmp_path / "absent.bin"))
