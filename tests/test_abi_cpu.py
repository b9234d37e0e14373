"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/srn.h declares, and its host-only entry points validate input."""
import ctypes as ct
import os
import re
import subprocess

import pytest

from paper_2308_02494_gb300 import build as pb
from paper_2308_02494_gb300 import srn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pb.build()   # incremental: recompiles only sources newer than their objects
    return srn.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "srn.h")).read()
    return sorted(set(re.findall(r"^(?:srn_status|const char\*)\s+(srn_\w+)\(", text, re.M)))


def test_header_and_binding_agree():
    assert _declared() == sorted(srn.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pb.LIB], capture_output=True, text=True).stdout
    names = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared():
        assert name in names, name
        assert getattr(lib, name) is not None


def _cfg(**kw):
    base = dict(n_bricks=1, n_grids=64, channels=2, res=32, hidden=64, precision=srn.SRN_BF16,
                flat_top_p=10, density_eps=1e-8, lr_feat=1e-2, lr_xform=1e-3, beta1=0.9,
                beta2=0.99, adam_eps=1e-8)
    base.update(kw)
    return srn.Config(**base)


def test_layout_offsets_and_groups(lib):
    L = srn.srn_param_layout(_cfg(n_bricks=3))
    M, R, C, K = 64, 32, 2, 128
    assert L.size_F >= M * R ** 3 * C and L.size_W1 >= 64 * K and L.size_G >= M * 12
    for off in (L.off_F, L.off_W1, L.off_W2, L.off_w3, L.off_G, L.n_group_a, L.n_params):
        assert off % 64 == 0
    assert L.off_W1 == 3 * L.size_F
    assert L.n_group_a == L.off_G and L.n_params == L.off_G + 3 * L.size_G


def test_workspace_grows_with_points(lib):
    a = srn.srn_workspace_size(_cfg(), 1 << 10)
    b = srn.srn_workspace_size(_cfg(), 1 << 20)
    assert 0 < a < b and b % 256 == 0


@pytest.mark.parametrize("kw, status", [
    (dict(hidden=32), srn.SRN_ERR_UNSUPPORTED),
    (dict(channels=3), srn.SRN_ERR_UNSUPPORTED),
    (dict(n_grids=48), srn.SRN_ERR_UNSUPPORTED),          # K = 96
    (dict(res=1), srn.SRN_ERR_INVALID_ARG),
    (dict(res=65), srn.SRN_ERR_UNSUPPORTED),
    (dict(n_bricks=0), srn.SRN_ERR_INVALID_ARG),
    (dict(n_bricks=65), srn.SRN_ERR_INVALID_ARG),
    (dict(flat_top_p=0), srn.SRN_ERR_UNSUPPORTED),
    (dict(precision=7), srn.SRN_ERR_INVALID_ARG),
    (dict(beta2=1.0), srn.SRN_ERR_INVALID_ARG),
    (dict(density_eps=0.0), srn.SRN_ERR_INVALID_ARG),
])
def test_bad_configs_are_rejected_with_a_message(lib, kw, status):
    with pytest.raises(srn.SrnError) as e:
        srn.srn_param_layout(_cfg(**kw))
    assert e.value.status == status
    assert srn.srn_last_error()


def test_create_rejects_null_tensors_without_touching_the_gpu(lib):
    t = srn.Tensors(None, None, None, None, None, None)
    h = ct.c_void_p()
    st = lib.srn_create(ct.byref(_cfg()), ct.byref(t), None, 0, 16, ct.byref(h))
    assert st == srn.SRN_ERR_INVALID_ARG
    assert lib.srn_destroy(None) == srn.SRN_ERR_INVALID_ARG


def test_tiled_volume_size_pads_each_extent_to_whole_tiles(lib):
    # 4 x 4 x 4-voxel tiles of float32: ceil(d / 4) tiles per axis, 256 bytes per tile
    for dims, tiles in [((4, 4, 4), 1), ((5, 4, 4), 2), ((5, 6, 7), 8), ((1024, 1024, 1024), 256 ** 3),
                        ((2, 3, 9), 3), ((513, 2, 2), 129)]:
        assert srn.srn_tiled_volume_bytes(list(dims)) == 256 * tiles, dims


def test_tiled_volume_size_rejects_an_extent_below_two(lib):
    with pytest.raises(srn.SrnError) as e:
        srn.srn_tiled_volume_bytes([8, 1, 8])
    assert "dimension 1" in str(e.value)
