"""GPU hash-grid query and its adjoint against the oracle (condition-aware
1e-5 rule), plus the BF16-table error statement."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from tests._parity import assert_cond_close

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def _grid(oracle, log2_T, res=RES16, seed=1):
    n_ent = oracle.hash_entries(res, log2_T)
    return scenes.make_hashgrid(seed, n_ent, res, log2_T)


def _pos(seed, n, lo=0.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, 3)).astype(np.float32)


def _fwd_check(gpu, oracle, grid, pos):
    desc = api.hashgrid_desc(grid.res, grid.log2_T)
    h = api.query_hashgrid(desc, torch.from_numpy(grid.table).to(gpu), torch.from_numpy(pos).to(gpu))
    ref, ab = oracle.hash_fwd(grid.res, grid.log2_T, grid.table, pos, with_abs=True)
    return assert_cond_close(h.cpu().numpy(), ref, ab, what="h")


def test_query_matches_oracle(gpu, oracle):
    grid = _grid(oracle, 19)
    pos = _pos(0, 200_000)
    # edge positions: the cube faces, corners, just inside/outside, clamped
    pos[:12] = [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.5, 1, 0], [1e-7, 0.9999999, 0.5], [-0.1, 1.2, 0.3],
                [0.5, 0.5, 0.5], [0.25, 0.75, 0.125], [1.0, 1.0, 0.999999], [0, 1, 0], [0.3, -5, 7], [1 - 2**-24, 0, 1]]
    _fwd_check(gpu, oracle, grid, pos)


def test_query_various_layouts(gpu, oracle):
    for res, log2_T in [([1], 4), ([3, 7, 100], 10), (RES16[:8], 21), ([4096], 24)]:
        grid = _grid(oracle, log2_T, res=res, seed=len(res))
        _fwd_check(gpu, oracle, grid, _pos(len(res), 10_000, -0.05, 1.05))


def test_query_empty(gpu):
    desc = api.hashgrid_desc(RES16, 19)
    h = api.query_hashgrid(desc, torch.zeros(10, 4, device=gpu), torch.zeros(0, 3, device=gpu))
    assert h.shape == (0, 64)


def _bwd_check(gpu, oracle, grid, pos, dh):
    desc = api.hashgrid_desc(grid.res, grid.log2_T)
    g = torch.zeros(grid.table.shape, dtype=torch.float32, device=gpu)
    api.query_hashgrid_bwd(desc, torch.from_numpy(pos).to(gpu), torch.from_numpy(dh).to(gpu), g)
    ref, ab = oracle.hash_bwd(grid.res, grid.log2_T, 4, pos, dh, with_abs=True)
    return assert_cond_close(g.cpu().numpy(), ref, ab, what="grad_table")


def test_table_gradient_matches_oracle(gpu, oracle):
    grid = _grid(oracle, 19)
    pos = _pos(2, 300_000)
    dh = np.random.default_rng(3).normal(size=(300_000, 64)).astype(np.float32)
    _bwd_check(gpu, oracle, grid, pos, dh)


def test_table_gradient_accumulates(gpu, oracle):
    grid = _grid(oracle, 12, res=RES16[:6])
    desc = api.hashgrid_desc(grid.res, grid.log2_T)
    pos = _pos(4, 5000)
    dh = np.random.default_rng(5).normal(size=(5000, 24)).astype(np.float32)
    g = torch.ones(grid.table.shape, dtype=torch.float32, device=gpu)
    api.query_hashgrid_bwd(desc, torch.from_numpy(pos).to(gpu), torch.from_numpy(dh).to(gpu), g)
    ref, ab = oracle.hash_bwd(grid.res, grid.log2_T, 4, pos, dh, with_abs=True)
    assert_cond_close(g.cpu().numpy(), ref + 1.0, ab + 1.0, what="accumulated")


def test_bf16_table_error_statement(gpu, oracle):
    """BF16 table and output with FP32 arithmetic: state the error against
    the FP64 oracle evaluated on the FP32 table (no pass/fail beyond bounds
    that BF16 rounding (2^-9 relative) implies)."""
    grid = _grid(oracle, 19)
    pos = _pos(6, 100_000)
    t32 = torch.from_numpy(grid.table).to(gpu)
    desc = api.hashgrid_desc(grid.res, grid.log2_T, table_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    h = api.query_hashgrid(desc, t32.to(torch.bfloat16), torch.from_numpy(pos).to(gpu)).float().cpu().numpy()
    ref, ab = oracle.hash_fwd(grid.res, grid.log2_T, grid.table, pos, with_abs=True)
    rel = np.abs(h - ref) / (ab + 1e-30)
    print("BF16 table+output: max err/sum|terms| = %.3e, mean = %.3e" % (rel.max(), rel.mean()))
    assert rel.max() < 2 * 2.0 ** -8


def test_query_table_alignments(gpu, oracle):
    """A 16-byte-aligned (not 32) FP32 table takes the per-row kernel; both
    variants give the oracle's values."""
    grid = _grid(oracle, 14, res=RES16[:8])
    pos = _pos(9, 20_000)
    desc = api.hashgrid_desc(grid.res, grid.log2_T)
    ref, ab = oracle.hash_fwd(grid.res, grid.log2_T, grid.table, pos, with_abs=True)
    buf = torch.zeros(grid.table.size + 8, dtype=torch.float32, device=gpu)
    for shift in (0, 4):  # floats: 0 -> 32-byte aligned, 4 -> 16-byte aligned
        t = buf[shift:shift + grid.table.size].view(grid.table.shape)
        t.copy_(torch.from_numpy(grid.table).to(gpu))
        h = api.query_hashgrid(desc, t, torch.from_numpy(pos).to(gpu))
        assert_cond_close(h.cpu().numpy(), ref, ab, what="h (shift %d)" % shift)


def test_hashed_index_golden_on_device(gpu):
    # the device query reads the row the hand-derived spatial hash names: a
    # one-level grid (resolution 4096, T = 2^19, hashed) whose row r holds
    # (r, r + 1/2, -r, 1), queried exactly on each golden vertex (weight 1 on
    # that vertex, 0 on the other seven corners)
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hash_index.json")))
    res, log2_T = [g["res"]], g["log2_T"]
    n_ent = api.hashgrid_n_entries(res, log2_T)
    r = np.arange(n_ent, dtype=np.float32)
    table = np.stack([r, r + 0.5, -r, np.ones_like(r)], axis=1)
    pos = np.array([c["v"] for c in g["cases"]], dtype=np.float32) / np.float32(g["res"])
    desc = api.hashgrid_desc(res, log2_T)
    h = api.query_hashgrid(desc, torch.from_numpy(table).to(gpu), torch.from_numpy(pos).to(gpu)).cpu().numpy()
    for k, c in enumerate(g["cases"]):
        i = c["index"]
        assert h[k].tolist() == [float(i), i + 0.5, -float(i), 1.0], c
