"""Argument checks of the misfit driver (host side; nothing is launched)."""
import ctypes

import pytest

import synthetic


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _desc(P, shape=(64, 64, 64), scheme=None):
    nz, ny, nx = shape
    return P.make_desc(nx, ny, nz, P.OOCS_WAVE if scheme is None else scheme, synthetic.wave_star_coef(),
                       1 << 40, temporal_depth=1, slab_planes=nz)


def test_workspace_bytes(P):
    d = _desc(P)
    n = 64 ** 3
    # 40 segments x 2 fields at 16 bits / value, then K + 5 FP32 fields
    assert P.oocs_misfit_workspace_bytes(d, 400, 10, 16) == 2 * 40 * n * 2 + 15 * n * 4
    assert P.oocs_misfit_workspace_bytes(d, 401, 10, 0) == 2 * 41 * n * 4 + 15 * n * 4
    with pytest.raises(P.OOCSError):
        P.oocs_misfit_workspace_bytes(d, 0, 10, 16)


def _forward(P, desc, ws_bytes, zr=8, src=(32, 32, 32), ws=256):
    return P.oocs_misfit_forward(desc, 256, src, [1.0], zr, 256, 20, 10, 16, ws, ws_bytes, 256, 256)


def test_rejects_bad_arguments(P):
    d = _desc(P)
    need = P.oocs_misfit_workspace_bytes(d, 20, 10, 16)
    for kw in (dict(ws_bytes=need - 1), dict(ws_bytes=need, zr=2), dict(ws_bytes=need, src=(64, 0, 0)),
               dict(ws_bytes=need, ws=0), dict(ws_bytes=need, ws=264)):
        with pytest.raises(P.OOCSError) as e:
            _forward(P, d, **kw)
        assert e.value.status == 1
    with pytest.raises(P.OOCSError):
        _forward(P, _desc(P, scheme=P.OOCS_HEAT), need)
    with pytest.raises(P.OOCSError):
        P.oocs_misfit_backward(d, 256, (32, 32, 32), [1.0], 8, 256, 20, 10, 16, 256, need - 1, 256)
