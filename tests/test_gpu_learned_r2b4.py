"""One learned step at R2B4 L30 (20 480 cells, 30 720 edges) with the
benchmark's hidden width of 512, element by element against the oracle's
learned step (oracle/corrector.py): FP64 dycores (4 reduced substeps, 5 in
the plain step), an untrained random network pair, inference in chunks of
8 192 rows (three chunks of cells and four of edges, the last ones ragged).

Every increment of w (interior half levels), exner, theta_v and vn must lie
within C = 12 root-sum-square estimates of the network output's error
(tests/mlp_bounds.py) scaled by the output statistics, with the input error
of the GPU's path (features in FP32, normalised in FP32, rounded to BF16)
propagated too; rho, the exner
history and w at the top and the ground are bitwise those of the reduced step."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state
from mlp_bounds import C, R, U32, forward_bound, init_params, rounded
from oracle import Dycore as OracleDycore, DycoreParams
from oracle import corrector as oc
from parity import to_torch, to_numpy

pytestmark = pytest.mark.gpu

NLEV, H, DT, CHUNK = 30, 512, 900.0, 8192


def _input_error(x, xm, xs, block_scale):
    """Per-element bound of the GPU's normalised BF16 input minus the oracle's
    normalised FP64 input: BF16 rounding, FP32 normalisation, FP32 features."""
    xn = (x - xm) / xs
    return R * np.abs(xn) + 4.0 * U32 * (np.abs(x) + np.abs(xm)) / xs + 2e-6 * block_scale / xs


def _block_scale(x, nlev, blocks):
    """Per-feature magnitude of its block (the velocity components share the zonal one's)."""
    out = np.empty(x.shape[1])
    for j, sj in enumerate(blocks):
        out[j * nlev:(j + 1) * nlev] = np.max(np.abs(x[:, sj * nlev:(sj + 1) * nlev]))
    return out


def test_learned_step_elementwise_r2b4_hidden_512(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z = make_grid(4), make_vct(NLEV)
    ored = OracleDycore(grid, z, DycoreParams(dtime=DT, ndyn_substeps=4))
    opl = OracleDycore(grid, z, DycoreParams(dtime=DT, ndyn_substeps=5))
    st = jw_type_state(grid, z, seed=6)
    st["exner_pr"] = ored.initial_exner_pr(st["exner"])
    sr_o = ored.step(st)
    cx = oc.column_features(ored, sr_o)
    ex = oc.edge_features(ored, sr_o, cx)
    ci, co, ei, eo = 5 * NLEV, 3 * NLEV - 1, 11 * NLEV, NLEV
    y_std_c = np.concatenate([np.full(NLEV - 1, 1e-3), np.full(NLEV, 1e-6), np.full(NLEV, 1e-3)])
    stats_c = tuple(np.asarray(a, np.float32) for a in (cx.mean(0), cx.std(0) + 1e-6, np.zeros(co), y_std_c))
    stats_e = tuple(np.asarray(a, np.float32) for a in (ex.mean(0), ex.std(0) + 1e-6, np.zeros(eo),
                                                         np.full(eo, 1e-2)))
    rng = np.random.default_rng(17)
    pc, pe = init_params(rng, ci, H, co), init_params(rng, ei, H, eo)
    prc, pre = rounded(pc, ci, H, co), rounded(pe, ei, H, eo)
    out_o, fb_o, r_o = oc.step_learned(ored, opl, (prc, (ci, H, co), stats_c), (pre, (ei, H, eo), stats_e), st,
                                       1e30)
    assert not fb_o

    G = P.Grid(grid)
    Rd = P.Dycore(G, z, dict(dtime=DT, ndyn_substeps=4))
    Pl = P.Dycore(G, z, dict(dtime=DT, ndyn_substeps=5))
    cn, en = P.MLP(ci, H, co, CHUNK), P.MLP(ei, H, eo, CHUNK)
    cn.set_params(pc)
    en.set_params(pe)
    cn.set_normalization(*stats_c)
    en.set_normalization(*stats_e)
    t = to_torch(st, cuda)
    tr = {k: v.clone() for k, v in t.items()}
    Rd.step(tr)
    fb, r = P.step_learned(Rd, Pl, cn, en, t, 1e30)
    assert not fb
    g, gr = to_numpy(t), to_numpy(tr)
    assert np.array_equal(g["rho"], gr["rho"]) and np.array_equal(g["exner_pr"], gr["exner_pr"])
    assert np.array_equal(g["w"][:, [0, -1]], gr["w"][:, [0, -1]])

    # output bounds of both networks on the oracle's normalised features
    bounds = {}
    for name, x, stats, pr, dims, blocks in (
            ("col", cx, stats_c, prc, (ci, H, co), [0, 1, 2, 3, 3]),
            ("edge", ex, stats_e, pre, (ei, H, eo), [0, 1, 2, 3, 3, 5, 6, 7, 8, 8, 10])):
        xm, xs, ym, ys = [np.asarray(a, np.float64) for a in stats]
        e_x = _input_error(x, xm, xs, _block_scale(x, NLEV, blocks))
        _, e_y = forward_bound(pr, (x - xm) / xs, *dims, ex=e_x)
        bounds[name] = e_y * ys
    bc, be = bounds["col"], bounds["edge"]
    pieces = (("w", np.s_[:, 1:-1], bc[:, :NLEV - 1]), ("exner", np.s_[:, :], bc[:, NLEV - 1:2 * NLEV - 1]),
              ("theta_v", np.s_[:, :], bc[:, 2 * NLEV - 1:]), ("vn", np.s_[:, :], be))
    for k, sl, b in pieces:
        inc = g[k][sl] - gr[k][sl]
        inc_o = out_o[k][sl] - sr_o[k][sl]
        # plus the FP32 increment's own rounding and the FP64 addition to the state
        tol = C * b + 2.0 * U32 * np.abs(inc_o) + 4.0 * 2.0 ** -52 * np.abs(gr[k][sl])
        excess = np.abs(inc - inc_o) - tol
        assert excess.max() <= 0.0, (k, float(excess.max()))
        assert np.median(C * b / (np.abs(inc_o) + 1e-300)) < 0.2, k
    assert r == pytest.approx(r_o, rel=3e-2)
    for x in (cn, en, Rd, Pl):
        x.close()
    G.close()
