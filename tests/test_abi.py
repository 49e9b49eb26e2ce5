"""The C-ABI library loads and exports every symbol include/inpc.h declares,
and its host-only entry points (size queries, argument validation) behave
as documented.  No compute calls: runs without a GPU."""
import os
import re

import pytest

from paper_2403_16862_gb300 import build, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    build.build()
    from paper_2403_16862_gb300 import _binding
    _binding.load()
    return _binding


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "inpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(inpc_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(B):
    import ctypes
    declared = _declared_functions()
    assert sorted(B.DECLARED) == declared
    lib = ctypes.CDLL(B.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert "sm_103a" in B.version()


def test_hashgrid_entries_match_layout_rule(B, oracle):
    from paper_2403_16862_gb300 import api
    for log2_T in (12, 19, 21):
        res = scenes.geometric_resolutions(16, 16, 4096)
        assert api.hashgrid_n_entries(res, log2_T) == oracle.hash_entries(res, log2_T)
    assert api.hashgrid_n_entries([1, 2, 3], 10) == oracle.hash_entries([1, 2, 3], 10)


def test_workspace_sizes(B):
    from paper_2403_16862_gb300 import api
    s1 = B.inpc_sample_workspace_size(65536, 1 << 22)
    s2 = B.inpc_sample_workspace_size(1 << 20, 1 << 24)
    assert 65536 * 16 <= s1 < s2
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900, 900, 640, 416, 1280, 832)
    opts = api.RasterOptions(n_channels=64, head_mode=True)
    w = api.rasterize_workspace_size(cam, opts, 1 << 22)
    assert w >= (1 << 22) * 4 * 8
    assert s1 % 256 == 0 and w % 256 == 0


def test_fused_backward_defers_fine_levels_of_large_tables(B):
    # The fused backward's fine half (levels 8..15 of 16) reduces in place
    # while its gradient rows fit the 64 MB L2 budget (2^19 rows of 16 B per
    # level: 64 MB); larger tables store those levels' rows, 16 B per point
    # and level, for the level-grouped pass: the workspace grows by that
    # buffer, 256-byte aligned.
    from paper_2403_16862_gb300 import api
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900, 900, 640, 416, 1280, 832)
    opts = api.RasterOptions(n_channels=64, head_mode=True)
    res = scenes.geometric_resolutions(16, 16, 4096)
    n = 1 << 20 | 3
    base = api.rasterize_bwd_hashgrid_workspace_size(cam, opts, api.hashgrid_desc(res, 19), n)
    assert base == api.rasterize_workspace_size(cam, opts, n)
    for log2_T in (20, 21):
        big = api.rasterize_bwd_hashgrid_workspace_size(cam, opts, api.hashgrid_desc(res, log2_T), n)
        assert big == (base + 255) // 256 * 256 + n * 8 * 16, log2_T


def test_argument_errors_are_reported(B):
    from paper_2403_16862_gb300 import api
    with pytest.raises(B.InpcError) as e:
        B.inpc_sample_workspace_size(0, 10)
    assert e.value.status == B.INPC_ERR_CAPACITY
    with pytest.raises(B.InpcError) as e:
        B.inpc_sample_workspace_size(1 << 25, 10)
    assert e.value.status == B.INPC_ERR_CAPACITY
    d = api.hashgrid_desc([16, 32], 10, n_feats=2)
    with pytest.raises(B.InpcError) as e:
        B.inpc_hashgrid_n_entries(d)
    assert e.value.status == B.INPC_ERR_UNSUPPORTED
    d = api.hashgrid_desc([16, 32], 30)
    with pytest.raises(B.InpcError) as e:
        B.inpc_hashgrid_n_entries(d)
    assert e.value.status == B.INPC_ERR_INVALID_ARG
    # the calibration's region must be a power of two of rows in range, and
    # its buffer 16-byte aligned (checked before anything touches a device)
    for rows, buf in ((3 << 12, 1 << 20), (1 << 9, 1 << 20), (1 << 27, 1 << 20), (1 << 16, (1 << 20) + 4)):
        with pytest.raises(B.InpcError) as e:
            B.inpc_l2_reduction_rate(buf, rows, False, None)
        assert e.value.status == B.INPC_ERR_INVALID_ARG, rows
    # null pointers are rejected before anything touches a device
    d = api.hashgrid_desc([16, 32], 10)
    with pytest.raises(B.InpcError) as e:
        B.inpc_query_hashgrid(d, None, None, 5, None, None)
    assert e.value.status == B.INPC_ERR_INVALID_ARG
    cam = scenes.make_camera((0, 0, -3), 10, 10, 5, 5, 10, 10)
    cc = api.camera(cam)
    with pytest.raises(B.InpcError) as e:
        B.inpc_rasterize_workspace_size(cc, api.RasterOptions(n_channels=200).c(), 10)
    assert e.value.status == B.INPC_ERR_UNSUPPORTED
    with pytest.raises(B.InpcError) as e:
        B.inpc_rasterize_workspace_size(cc, api.RasterOptions(n_channels=4, tile_w=32, tile_h=16).c(), 10)
    assert e.value.status == B.INPC_ERR_INVALID_ARG
    # the forward takes up to 2^28 points; beyond 2^25 the near plane's bits
    # are the depth field's base and the far plane must stay within 2^(56 - 26)
    # of them for 26-bit point indices
    o4 = api.RasterOptions(n_channels=4).c()
    assert B.inpc_rasterize_workspace_size(cc, o4, 1 << 28) > B.inpc_rasterize_workspace_size(cc, o4, 1 << 25)
    with pytest.raises(B.InpcError) as e:
        B.inpc_rasterize_workspace_size(cc, o4, (1 << 28) + 1)
    assert e.value.status == B.INPC_ERR_CAPACITY
    wide = api.camera(scenes.make_camera((0, 0, -3), 10, 10, 5, 5, 10, 10, near=1e-6, far=1e6))
    assert B.inpc_rasterize_workspace_size(wide, o4, 1 << 25) > 0
    with pytest.raises(B.InpcError) as e:
        B.inpc_rasterize_workspace_size(wide, o4, 1 << 28)
    assert e.value.status == B.INPC_ERR_CAPACITY
    # the calls that continue from the forward keep 25-bit point indices
    with pytest.raises(B.InpcError) as e:
        B.inpc_rasterize_bwd(cc, o4, None, None, None, (1 << 25) + 1, None, None, None, None, None, None, 0, None)
    assert e.value.status == B.INPC_ERR_CAPACITY
    with pytest.raises(B.InpcError) as e:
        B.inpc_rasterize_fwd(cc, api.RasterOptions(n_channels=4).c(), None, None, None, 10, None, None, None,
                             None, 0, None)
    assert e.value.status == B.INPC_ERR_INVALID_ARG
    assert "workspace" in str(e.value)


def test_render_batch_argument_errors(B):
    """inpc_render_batch validates its arguments before any stream work."""
    from paper_2403_16862_gb300 import api
    cam = scenes.make_camera((0, 0, -3), 10, 10, 5, 5, 10, 10)
    desc = api.hashgrid_desc(scenes.geometric_resolutions(16, 16, 4096), 14)
    tree = B.InpcOctree(1, 1, 1, 1.0, 8)  # never dereferenced: validation fails first
    job = B.InpcViewJob(cam=api.camera(cam), opts=api.RasterOptions(n_channels=64, head_mode=True).c(), view_id=0,
                        n_samples=10, d_image=1)
    cases = [
        (dict(table=0, jobs=[job], grad_table=1, streams=[1]), "null pointer"),
        (dict(table=1, jobs=[job], grad_table=1, streams=[]), "n_streams"),
        (dict(table=1, jobs=[job], grad_table=1, streams=[7, 7]), "repeats"),
        (dict(table=1, jobs=[job], grad_table=None, streams=[1]), "grad_table is null"),
    ]
    for kw, msg in cases:
        with pytest.raises(B.InpcError) as e:
            B.inpc_render_batch(tree, 0, desc, kw["table"], kw["jobs"], kw["grad_table"], kw["streams"])
        assert e.value.status == B.INPC_ERR_INVALID_ARG and msg in str(e.value), (msg, str(e.value))
    given = B.InpcViewJob(cam=api.camera(cam), opts=api.RasterOptions(n_channels=64).c(), n_samples=10)
    with pytest.raises(B.InpcError) as e:
        B.inpc_render_batch(tree, 0, desc, 1, [given], 1, [1])
    assert e.value.status == B.INPC_ERR_INVALID_ARG and "head mode" in str(e.value)
    B.inpc_render_batch(tree, 0, desc, 1, [], 1, [1])  # an empty batch is a no-op


def test_binding_constants_match_the_header(B):
    # the Python constants mirror the header's macros and enum values
    src = open(os.path.join(ROOT, "include", "inpc.h")).read()
    m = re.search(r"#define INPC_SAMPLE_STATIC_SCRATCH_BYTES \(\((\d+)u << 20\) \+ \((\d+)u << 10\)\)", src)
    assert m and B.INPC_SAMPLE_STATIC_SCRATCH_BYTES == (int(m.group(1)) << 20) + (int(m.group(2)) << 10)
    for name in ("INPC_DEV_BAD_WEIGHT", "INPC_DEV_NO_WEIGHT", "INPC_DEV_BAD_LEAF", "INPC_DEV_BAD_BLEND_WEIGHT"):
        v = re.search(r"#define %s (0x[0-9a-fA-F]+)u" % name, src)
        assert v and getattr(B, name) == int(v.group(1), 16), name
    for name in ("INPC_ERR_INVALID_ARG", "INPC_ERR_CUDA", "INPC_ERR_CAPACITY", "INPC_ERR_TIMEOUT",
                 "INPC_ERR_UNSUPPORTED"):
        v = re.search(r"%s = (\d+)" % name, src)
        assert v and getattr(B, name) == int(v.group(1)), name
