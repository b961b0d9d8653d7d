"""Checkpoint and restart (icon_dycore_save / icon_dycore_load): a run that
is saved, reloaded into fresh arrays and continued equals the uninterrupted
run bit for bit, in both precisions and from device or host arrays; a file of
another grid, a damaged or truncated file and a missing file are refused and
leave the state as it was."""
import os

import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu


def _bitwise_equal(a, b):
    return all(np.array_equal(a[k].view(np.uint64), b[k].view(np.uint64)) for k in a)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_restart_equals_uninterrupted_run(built_lib, cuda, tmp_path, precision):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(3, 30, 900.0, rayleigh=0.05, seed=6)
    prec = P.ICON_PREC_MIXED if precision == "mixed" else P.ICON_PREC_FP64
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op, rayleigh_coeff=0.05, precision=prec))
    t = to_torch(st, cuda)
    d.step(t)
    path = str(tmp_path / "state.ckpt")
    d.save(t, path)
    assert os.path.getsize(path) == 64 + 8 * sum(v.size for v in st.values())
    d.step(t)
    d.step(t)
    r = {k: torch.full_like(v, float("nan")) for k, v in t.items()}
    d.load(r, path)
    d.step(r)
    d.step(r)
    d.synchronize()
    assert _bitwise_equal(to_numpy(r), to_numpy(t))
    d.close()


def test_host_arrays_round_trip(built_lib, cuda, tmp_path):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0, seed=7)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    host = {k: np.ascontiguousarray(v) for k, v in st.items()}
    path = str(tmp_path / "host.ckpt")
    d.save(host, path)
    back = {k: np.full_like(v, np.nan) for k, v in host.items()}
    d.load(back, path)
    assert _bitwise_equal(back, host)
    # a device load of the same file gives the same numbers
    dev = {k: v.clone() for k, v in to_torch(st, cuda).items()}
    for v in dev.values():
        v.fill_(0.0)
    d.load(dev, path)
    assert _bitwise_equal(to_numpy(dev), host)
    d.close()


def test_bad_files_refused_and_state_kept(built_lib, cuda, tmp_path):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0, seed=8)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    t = to_torch(st, cuda)
    good = str(tmp_path / "good.ckpt")
    d.save(t, good)
    data = open(good, "rb").read()
    keep = to_numpy(t)

    damaged = str(tmp_path / "damaged.ckpt")
    b = bytearray(data)
    b[64 + 8 * 1000 + 3] ^= 0x10          # one bit of one value of vn
    open(damaged, "wb").write(bytes(b))
    truncated = str(tmp_path / "truncated.ckpt")
    open(truncated, "wb").write(data[:-8])
    foreign = str(tmp_path / "foreign.ckpt")
    b = bytearray(data)
    b[12] ^= 0x01                          # nlev in the header
    open(foreign, "wb").write(bytes(b))
    for bad in (damaged, truncated, foreign, str(tmp_path / "missing.ckpt")):
        with pytest.raises(P.IconError):
            d.load(t, bad)
        assert _bitwise_equal(to_numpy(t), keep), bad
    # a dycore with another number of levels refuses the good file too
    grid2, z2, op2, od2, st2 = setup(2, 20, 1800.0, seed=8)
    d2 = P.Dycore(g, z2, gpu_params(op2))
    t2 = to_torch(st2, cuda)
    with pytest.raises(P.IconError):
        d2.load(t2, good)
    d2.close()
    d.close()
