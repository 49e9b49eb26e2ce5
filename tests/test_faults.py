"""Host-side fault injection (inpc_set_fault / INPC_FAULT): every failure is
made on the host, none on a GPU.

* workspace_overflow: every workspace-size query reports INPC_ERR_CAPACITY.
* corrupt_args: every compute entry point sees its first array argument as
  NULL and must return INPC_ERR_INVALID_ARG from its own validation, before
  it enqueues anything; repeated failing calls leak no host memory.
* queue_short (a GPU test in test_gpu_batch_front.py): a persistent batch
  launch waits for a producer that never comes; the wait runs out.

The corrupt_args calls pass made-up device addresses for the other arrays:
they are never dereferenced when validation works, but a call whose
validation missed the corrupted argument would launch a kernel on them, so
that check runs only where no CUDA device is present."""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_2403_16862_gb300 import build, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    build.build()
    from paper_2403_16862_gb300 import _binding
    _binding.load()
    yield _binding
    _binding.inpc_set_fault(None)


def _cpu_only():
    import torch
    if torch.cuda.is_available():
        pytest.skip("made-up device addresses are only passed where no CUDA device exists")


def _structs(B):
    from paper_2403_16862_gb300 import api
    fake = 1 << 20  # a 256-byte aligned made-up address, never dereferenced
    tree = B.InpcOctree(fake, fake, fake, 1.0, 4096)
    cam = api.camera(scenes.make_camera((0.5, 0.5, -1.2), 100.0, 100.0, 32.0, 32.0, 64, 64))
    opts = api.RasterOptions(n_channels=64, head_mode=True).c()
    opts_given = api.RasterOptions(n_channels=8).c()
    desc = api.hashgrid_desc(scenes.geometric_resolutions(16, 16, 4096), 19)
    return fake, tree, cam, opts, opts_given, desc


def _calls(B):
    """Every compute entry point, with valid-looking arguments."""
    fake, tree, cam, opts, opts_given, desc = _structs(B)
    big = 1 << 40
    job = B.InpcViewJob(cam=cam, opts=opts, view_id=0, n_samples=1000, leaf_idx=fake, pos=fake, h=fake, image=fake,
                        T_final=fake, n_contrib=fake, d_image=fake, sample_ws=fake, sample_ws_bytes=big,
                        raster_ws=fake, raster_ws_bytes=big)
    fv = B.InpcFrontView(view_id=0, n_samples=1000, leaf_idx=fake, pos=fake, h=fake)
    return {
        "inpc_sample_octree": lambda: B.inpc_sample_octree(tree, 0, 0, 1000, fake, fake, None, fake, big, None),
        "inpc_sample_octree_noalloc": lambda: B.inpc_sample_octree_noalloc(tree, 0, 0, 1000, fake, fake, None, None),
        "inpc_sample_octree_halton": lambda: B.inpc_sample_octree_halton(tree, 0, 1000, fake, fake, None, fake, big,
                                                                         None),
        "inpc_sample_octree_view": lambda: B.inpc_sample_octree_view(tree, cam, 0, 0, 1000, 4, fake, fake, None, fake,
                                                                     big, None),
        "inpc_view_weights": lambda: B.inpc_view_weights(tree, cam, 0.5, 1e-8, fake, None),
        "inpc_level_weights": lambda: B.inpc_level_weights(tree, 0.5, fake, None),
        "inpc_philox4x32_10": lambda: B.inpc_philox4x32_10(fake, fake, 10, fake, None),
        "inpc_accumulate_image": lambda: B.inpc_accumulate_image(fake, B.INPC_F32, 100, 0.5, fake, None),
        "inpc_query_hashgrid": lambda: B.inpc_query_hashgrid(desc, fake, fake, 1000, fake, None),
        "inpc_query_hashgrid_bwd": lambda: B.inpc_query_hashgrid_bwd(desc, fake, fake, 1000, fake, None),
        "inpc_rasterize_fwd": lambda: B.inpc_rasterize_fwd(cam, opts, fake, None, fake, 1000, fake, fake, fake, fake,
                                                           big, None),
        "inpc_rasterize_bwd": lambda: B.inpc_rasterize_bwd(cam, opts_given, fake, fake, fake, 1000, fake, fake, fake,
                                                           fake, fake, fake, big, None),
        "inpc_rasterize_bwd_hashgrid": lambda: B.inpc_rasterize_bwd_hashgrid(cam, opts, desc, fake, fake, 1000, fake,
                                                                             fake, fake, fake, None, fake, big, None),
        "inpc_rasterize_point_weights": lambda: B.inpc_rasterize_point_weights(cam, opts, fake, 1000, fake, fake,
                                                                               fake, big, None),
        "inpc_octree_update": lambda: B.inpc_octree_update(fake, fake, 1000, fake, fake, 4096, 0.9, fake, big, None),
        "inpc_octree_subdivide": lambda: B.inpc_octree_subdivide(tree, fake, 0.5, 1 << 24, fake, fake, fake, fake,
                                                                 1 << 16, fake, big, None),
        "inpc_octree_prune": lambda: B.inpc_octree_prune(tree, fake, 0.01, fake, fake, fake, fake, 1 << 16, fake, big,
                                                         None),
        "inpc_contract_positions": lambda: B.inpc_contract_positions(fake, 1000, (0.0, 0.0, 0.0), 1.0, fake, None),
        "inpc_sh_head_fwd": lambda: B.inpc_sh_head_fwd(cam, fake, fake, B.INPC_F32, 1000, 40, fake, fake, None),
        "inpc_sh_head_bwd": lambda: B.inpc_sh_head_bwd(cam, fake, fake, B.INPC_F32, 1000, 40, fake, fake, fake, None),
        "inpc_render_batch": lambda: B.inpc_render_batch(tree, 0, desc, fake, [job], fake, [fake]),
        "inpc_render_batch_persistent": lambda: B.inpc_render_batch_persistent(tree, 0, desc, fake, [job], fake,
                                                                               [fake], fake, big, 1000),
        "inpc_sample_query_batch": lambda: B.inpc_sample_query_batch(tree, 0, desc, fake, [fv], 1000, fake, big,
                                                                     None),
        "inpc_l2_reduction_rate": lambda: B.inpc_l2_reduction_rate(fake, 1 << 16, False, None),
    }


def _size_queries(B):
    _, _, cam, opts, _, desc = _structs(B)
    return {
        "inpc_sample_workspace_size": lambda: B.inpc_sample_workspace_size(4096, 1000),
        "inpc_rasterize_workspace_size": lambda: B.inpc_rasterize_workspace_size(cam, opts, 1000),
        "inpc_rasterize_bwd_hashgrid_workspace_size": lambda: B.inpc_rasterize_bwd_hashgrid_workspace_size(
            cam, opts, desc, 1000),
        "inpc_octree_update_workspace_size": lambda: B.inpc_octree_update_workspace_size(4096),
        "inpc_octree_refine_workspace_size": lambda: B.inpc_octree_refine_workspace_size(4096),
        "inpc_sample_query_batch_workspace_size": lambda: B.inpc_sample_query_batch_workspace_size(4096, 3),
    }


def test_every_compute_entry_is_covered(B):
    # the table of calls names every compute entry point of the header
    from tests.test_abi import _declared_functions
    host_only = {"inpc_last_error", "inpc_version", "inpc_kernel_launches", "inpc_read_device_status",
                 "inpc_kernel_timer_enable", "inpc_kernel_timer_read", "inpc_hashgrid_n_entries", "inpc_set_fault"}
    sizes = {n for n in _declared_functions() if n.endswith("_workspace_size")}
    assert set(_calls(B)) == set(_declared_functions()) - host_only - sizes
    assert set(_size_queries(B)) == sizes


def test_workspace_overflow_injection(B):
    sizes = _size_queries(B)
    for name, q in sizes.items():
        assert q() > 0, name
    B.inpc_set_fault("workspace_overflow")
    try:
        for name, q in sizes.items():
            with pytest.raises(B.InpcError) as e:
                q()
            assert e.value.status == B.INPC_ERR_CAPACITY and "injected" in str(e.value), name
    finally:
        B.inpc_set_fault(None)
    for name, q in sizes.items():
        assert q() > 0, name


def test_corrupt_args_injection_is_caught_by_validation(B):
    _cpu_only()
    calls = _calls(B)
    B.inpc_set_fault("corrupt_args")
    try:
        for name, call in calls.items():
            with pytest.raises(B.InpcError) as e:
                call()
            assert e.value.status == B.INPC_ERR_INVALID_ARG, (name, str(e.value))
    finally:
        B.inpc_set_fault(None)


def _rss_kb():
    with open("/proc/self/status") as f:
        for line in f:
            if line.startswith("VmRSS:"):
                return int(line.split()[1])
    return 0


def test_failing_calls_leak_nothing(B):
    _cpu_only()
    calls = list(_calls(B).values())
    B.inpc_set_fault("corrupt_args")
    try:
        for call in calls * 20:  # warm up allocator pools and message buffers
            with pytest.raises(B.InpcError):
                call()
        before = _rss_kb()
        for call in calls * 400:
            with pytest.raises(B.InpcError):
                call()
        grown = _rss_kb() - before
    finally:
        B.inpc_set_fault(None)
    assert grown < 2048, "host memory grew by %d kB over %d failing calls" % (grown, 400 * len(calls))


def test_unknown_fault_is_rejected(B):
    with pytest.raises(B.InpcError) as e:
        B.inpc_set_fault("no_such_fault")
    assert e.value.status == B.INPC_ERR_INVALID_ARG
    B.inpc_set_fault("")


def test_environment_variable_arms_a_fault():
    code = ("from paper_2403_16862_gb300 import _binding as B\n"
            "try:\n"
            "    B.inpc_sample_workspace_size(4096, 10)\n"
            "except B.InpcError as e:\n"
            "    raise SystemExit(0 if e.status == B.INPC_ERR_CAPACITY else 2)\n"
            "raise SystemExit(1)\n")
    env = dict(os.environ, INPC_FAULT="workspace_overflow")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
