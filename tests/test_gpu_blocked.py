"""ICON nproma-blocked state arrays (Fortran X(nproma, nlev_x, nblks)) through
the C-ABI: the conversion matches the layout definition written out with numpy
reshapes, round trips bit for bit, leaves pad points alone, and a step of the
blocked state equals the step of the same state in the library's layout."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch

pytestmark = pytest.mark.gpu

FIELDS = ("vn", "w", "rho", "exner", "theta_v", "exner_pr")


def blocked_reference(x, nproma):
    """(n, nlev_x) level-contiguous -> C array (nblks, nlev_x, nproma), i.e. the
    Fortran array X(nproma, nlev_x, nblks); pads NaN."""
    n, nl = x.shape
    nb = -(-n // nproma)
    pad = np.full((nb * nproma, nl), np.nan)
    pad[:n] = x
    return pad.reshape(nb, nproma, nl).transpose(0, 2, 1).copy()


@pytest.mark.parametrize("nproma", [32, 37, 1])
def test_blocked_conversion_matches_layout_and_round_trips(built_lib, cuda, nproma):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op, synchronous=1))
    t = to_torch(st, cuda)
    ref = {k: blocked_reference(st[k], nproma) for k in FIELDS}
    sentinel = -12345.0
    blk = {k: torch.full(ref[k].shape, sentinel, dtype=torch.float64, device=cuda) for k in FIELDS}
    d.to_blocked(nproma, t, blk)
    for k in FIELDS:
        got = blk[k].cpu().numpy()
        mask = ~np.isnan(ref[k])
        assert np.array_equal(got[mask], ref[k][mask]), k
        assert np.all(got[~mask] == sentinel), k   # pads untouched
    back = {k: torch.empty_like(t[k]) for k in FIELDS}
    d.from_blocked(nproma, blk, back)
    assert all(torch.equal(back[k], t[k]) for k in FIELDS)


def test_step_of_blocked_state_equals_step(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    nproma = 40
    grid, z, op, od, st = setup(2, 30, 1800.0, rayleigh=0.05)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op, rayleigh_coeff=0.05, synchronous=1))
    t = to_torch(st, cuda)
    blk = {k: torch.from_numpy(np.nan_to_num(blocked_reference(st[k], nproma))).to(cuda) for k in FIELDS}
    d.step_blocked(nproma, blk)
    d.step(t)
    back = {k: torch.empty_like(t[k]) for k in FIELDS}
    d.from_blocked(nproma, blk, back)
    assert all(torch.equal(back[k], t[k]) for k in FIELDS)


def test_blocked_argument_errors(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(1, 10, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    t = to_torch(st, cuda)
    other = {k: torch.empty_like(v) for k, v in t.items()}
    for bad in (0, -3):
        with pytest.raises(P.IconError) as e:
            d.to_blocked(bad, t, other)
        assert e.value.code == P.ICON_ERR_ARG
    with pytest.raises(P.IconError) as e:   # destination aliases the source
        d.to_blocked(8, t, dict(other, rho=t["rho"]))
    assert e.value.code == P.ICON_ERR_ARG
    host = {k: v.cpu().numpy() for k, v in t.items()}
    with pytest.raises(P.IconError) as e:
        d.from_blocked(8, host, other)
    assert e.value.code == P.ICON_ERR_ARG
