"""Learned corrector on the GPU, through the C-ABI: features and targets
against the FP64 oracle, a whole learned step against the oracle's, the
fallback to the plain step, rho untouched, invariance to the inference chunk
size, argument errors, and the gain of a corrector trained on the GPU on
held-out seeds."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state
from oracle import Dycore as OracleDycore, DycoreParams
from oracle import corrector as oc
from parity import to_torch, to_numpy

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as the GPU stores weights."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _state(grid, z, seed, ex_ref):
    st = jw_type_state(grid, z, seed=seed)
    st["exner_pr"] = st["exner"] - ex_ref[None, :]
    return st


def _block_rel(a, b, nlev, scale_of):
    """Largest per-block max-norm difference of two [n, nblocks nlev] arrays, each
    block relative to the magnitude of the block scale_of[j] (the velocity
    components are sums of FP32 terms of the size of vn, so both are measured
    against the zonal component's scale)."""
    out = 0.0
    for j, sj in enumerate(scale_of):
        x, y = a[:, j * nlev:(j + 1) * nlev], b[:, j * nlev:(j + 1) * nlev]
        scale = np.max(np.abs(b[:, sj * nlev:(sj + 1) * nlev]))
        out = max(out, float(np.max(np.abs(x - y)) / max(scale, 1e-300)))
    return out


def test_features_match_oracle(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    nlev = 30
    grid, z = make_grid(3), make_vct(nlev)
    od = OracleDycore(grid, z, DycoreParams(dtime=900.0))
    st = _state(grid, z, 4, od.reference_state()[1])
    G = P.Grid(grid)
    D = P.Dycore(G, z, dict(dtime=900.0))
    t = to_torch(st, cuda)
    cx = torch.empty((grid.n_cells, 5 * nlev), dtype=torch.float32, device=cuda)
    ex = torch.empty((grid.n_edges, 11 * nlev), dtype=torch.float32, device=cuda)
    D.corrector_features(t, cx, ex)
    D.synchronize()
    ocx = oc.column_features(od, st)
    oex = oc.edge_features(od, st, ocx)
    assert _block_rel(cx.cpu().numpy().astype(np.float64), ocx, nlev, [0, 1, 2, 3, 3]) < 2e-6
    assert _block_rel(ex.cpu().numpy().astype(np.float64), oex, nlev, [0, 1, 2, 3, 3, 5, 6, 7, 8, 8, 10]) < 2e-6


def test_targets_are_the_rounded_difference_of_the_two_steps(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    nlev = 30
    grid, z = make_grid(2), make_vct(nlev)
    G = P.Grid(grid)
    R = P.Dycore(G, z, dict(dtime=900.0, ndyn_substeps=4))
    Pl = P.Dycore(G, z, dict(dtime=900.0, ndyn_substeps=5))
    st = to_torch(_state(grid, z, 1, R.reference_state()[1]), cuda)
    sr = {k: v.clone() for k, v in st.items()}
    sp = {k: v.clone() for k, v in st.items()}
    R.step(sr)
    Pl.step(sp)
    cy = torch.empty((grid.n_cells, 3 * nlev - 1), dtype=torch.float32, device=cuda)
    ey = torch.empty((grid.n_edges, nlev), dtype=torch.float32, device=cuda)
    R.corrector_targets(sr, sp, cy, ey)
    R.synchronize()
    ocy, oey = oc.targets(to_numpy(sr), to_numpy(sp))
    assert np.array_equal(cy.cpu().numpy(), ocy.astype(np.float32))
    assert np.array_equal(ey.cpu().numpy(), oey.astype(np.float32))
    assert float(ey.abs().max()) > 0.0


def _random_net(rng, n_in, n_hid, n_out):
    parts = [rng.standard_normal((n_hid, n_in)) / np.sqrt(n_in), 0.1 * rng.standard_normal(n_hid),
             rng.standard_normal((n_hid, n_hid)) / np.sqrt(n_hid), 0.1 * rng.standard_normal(n_hid),
             rng.standard_normal((n_out, n_hid)) / np.sqrt(n_hid), 0.1 * rng.standard_normal(n_out)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def _rounded(p, n_in, n_hid, n_out):
    from oracle import mlp as omlp
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, n_in, n_hid, n_out)
    return np.concatenate([bf16(W1).ravel(), b1, bf16(W2).ravel(), b2, bf16(W3).ravel(), b3])


def test_learned_step_matches_oracle(built_lib, cuda):
    """FP64 dycores, one learned step of an untrained (random) network pair on
    the GPU and in the oracle: the increments agree to the BF16 network's
    precision, rho is bitwise the reduced step's, and the check values agree."""
    import paper_2608_21150_gb300 as P
    nlev, H = 30, 64
    grid, z = make_grid(2), make_vct(nlev)
    ored = OracleDycore(grid, z, DycoreParams(dtime=900.0, ndyn_substeps=4))
    opl = OracleDycore(grid, z, DycoreParams(dtime=900.0, ndyn_substeps=5))
    st = _state(grid, z, 2, ored.reference_state()[1])
    sr_o = ored.step(st)
    cx = oc.column_features(ored, sr_o)
    ex = oc.edge_features(ored, sr_o, cx)
    ci, co, ei, eo = 5 * nlev, 3 * nlev - 1, 11 * nlev, nlev
    y_std_c = np.concatenate([np.full(nlev - 1, 1e-3), np.full(nlev, 1e-6), np.full(nlev, 1e-3)])
    stats_c = (cx.mean(0), cx.std(0) + 1e-6, np.zeros(co), y_std_c)
    stats_e = (ex.mean(0), ex.std(0) + 1e-6, np.zeros(eo), np.full(eo, 1e-2))
    stats_c = tuple(np.asarray(a, dtype=np.float32) for a in stats_c)
    stats_e = tuple(np.asarray(a, dtype=np.float32) for a in stats_e)
    rng = np.random.default_rng(7)
    pc, pe = _random_net(rng, ci, H, co), _random_net(rng, ei, H, eo)
    out_o, fb_o, r_o = oc.step_learned(ored, opl, (_rounded(pc, ci, H, co), (ci, H, co), stats_c),
                                       (_rounded(pe, ei, H, eo), (ei, H, eo), stats_e), st, 1e30)
    assert not fb_o
    G = P.Grid(grid)
    R = P.Dycore(G, z, dict(dtime=900.0, ndyn_substeps=4))
    Pl = P.Dycore(G, z, dict(dtime=900.0, ndyn_substeps=5))
    cn, en = P.MLP(ci, H, co, 1024), P.MLP(ei, H, eo, 1024)   # two chunks of cells and of edges
    cn.set_params(pc)
    en.set_params(pe)
    cn.set_normalization(*stats_c)
    en.set_normalization(*stats_e)
    t = to_torch(st, cuda)
    tr = {k: v.clone() for k, v in t.items()}
    R.step(tr)
    fb, r = P.step_learned(R, Pl, cn, en, t, 1e30)
    assert not fb
    g, gr = to_numpy(t), to_numpy(tr)
    assert np.array_equal(g["rho"], gr["rho"]) and np.array_equal(g["exner_pr"], gr["exner_pr"])
    assert np.array_equal(g["w"][:, [0, -1]], gr["w"][:, [0, -1]])
    for k, sl in (("vn", np.s_[:, :]), ("w", np.s_[:, 1:-1]), ("exner", np.s_[:, :]), ("theta_v", np.s_[:, :])):
        inc = g[k][sl] - gr[k][sl]
        inc_o = out_o[k][sl] - sr_o[k][sl]
        rel = np.linalg.norm(inc - inc_o) / np.linalg.norm(inc_o)
        assert rel < 3e-2, (k, rel)
    assert r == pytest.approx(r_o, rel=3e-2)


# ---------------------------------------------------------------------------
# a corrector trained on the GPU (R2B4 L30, 4 vs 5 substeps, mixed precision)

NLEV, DT, BIS = 30, 1440.0, 4


@pytest.fixture(scope="module")
def trained(built_lib):
    import torch
    import paper_2608_21150_gb300 as P
    from paper_2608_21150_gb300 import corrector as C
    dev = torch.device("cuda", 0)
    grid, z = make_grid(BIS), make_vct(NLEV)
    G = P.Grid(grid)
    base = dict(dtime=DT, rayleigh_coeff=0.05, precision=P.ICON_PREC_MIXED)
    R = P.Dycore(G, z, dict(base, ndyn_substeps=4))
    Pl = P.Dycore(G, z, dict(base, ndyn_substeps=5))
    ex_ref = R.reference_state()[1]
    data = C.Dataset()
    for seed in (0, 1, 2, 3):
        st = to_torch(_state(grid, z, seed, ex_ref), dev)
        for _ in range(10):
            Pl.step(st)
        for _ in range(10):
            st = C.add_pair(R, Pl, st, data)
            for _ in range(2):
                Pl.step(st)
    cx, cy, ex, ey = data.cat()
    cn, en = C.make_nets(NLEV, hidden=256, max_batch=2048, seed=1)
    lc = C.fit(cn, cx, cy, NLEV, 1500, batch=1024, lr=1e-3)
    le = C.fit(en, ex, ey, NLEV, 1500, batch=1024, lr=1e-3)
    return dict(P=P, C=C, dev=dev, grid=grid, z=z, G=G, R=R, Pl=Pl, cn=cn, en=en, ex_ref=ex_ref,
                losses=(lc, le))


def _spun_up(tr, seed, steps=10):
    st = to_torch(_state(tr["grid"], tr["z"], seed, tr["ex_ref"]), tr["dev"])
    for _ in range(steps):
        tr["Pl"].step(st)
    return st


def test_training_reduces_the_loss(trained):
    for losses in trained["losses"]:
        assert np.mean(losses[-50:]) < 0.5 * np.mean(losses[:10])


def test_trained_corrector_reduces_the_error_on_held_out_seeds(trained):
    P, C, R, Pl = trained["P"], trained["C"], trained["R"], trained["Pl"]
    ratios = {k: [] for k in ("vn", "w", "exner", "theta_v")}
    for seed in (10, 11):
        st = _spun_up(trained, seed)
        for _ in range(10):
            sp, sr, sl = C.clone_state(st), C.clone_state(st), C.clone_state(st)
            Pl.step(sp)
            R.step(sr)
            fb, r = P.step_learned(R, Pl, trained["cn"], trained["en"], sl, 3.0)
            assert not fb and r < 3.0
            er, el = C.field_errors(sr, sp), C.field_errors(sl, sp)
            for k in ratios:
                ratios[k].append(el[k] / er[k])
            assert torch_equal(sl["rho"], sr["rho"])
            st = sp
            for _ in range(2):
                Pl.step(st)
    mean = {k: float(np.mean(v)) for k, v in ratios.items()}
    assert all(m < 0.6 for m in mean.values()), mean


def test_rejected_correction_is_the_plain_step_bitwise(trained):
    P, C = trained["P"], trained["C"]
    st = _spun_up(trained, 12)
    sp, sl = C.clone_state(st), C.clone_state(st)
    trained["Pl"].step(sp)
    fb, r = P.step_learned(trained["R"], trained["Pl"], trained["cn"], trained["en"], sl, 0.0)
    assert fb and r > 0.0
    assert all(torch_equal(sl[k], sp[k]) for k in sl)


def torch_equal(a, b):
    import torch
    return torch.equal(a, b)


def test_out_of_distribution_state_falls_back(trained):
    """The unbalanced initial state (before any adjustment step) is far from the
    training distribution: the check rejects the correction."""
    P, C = trained["P"], trained["C"]
    st = to_torch(_state(trained["grid"], trained["z"], 13, trained["ex_ref"]), trained["dev"])
    sp = C.clone_state(st)
    trained["Pl"].step(sp)
    fb, r = P.step_learned(trained["R"], trained["Pl"], trained["cn"], trained["en"], st, 3.0)
    assert fb and r > 3.0
    assert all(torch_equal(st[k], sp[k]) for k in st)


def test_non_finite_rho_falls_back(trained):
    P, C = trained["P"], trained["C"]
    st = _spun_up(trained, 14, steps=2)
    st["rho"][5, 3] = float("nan")
    fb, r = P.step_learned(trained["R"], trained["Pl"], trained["cn"], trained["en"], st, 3.0)
    assert fb and np.isnan(r)


def test_result_does_not_depend_on_the_chunk_size(trained):
    P, C = trained["P"], trained["C"]
    cn, en = trained["cn"], trained["en"]
    c2 = P.MLP(cn.n_in, cn.n_hidden, cn.n_out, 960)
    e2 = P.MLP(en.n_in, en.n_hidden, en.n_out, 960)
    for a, b in ((cn, c2), (en, e2)):
        b.set_params(a.params())
        b.set_normalization(*a.normalization)
    st = _spun_up(trained, 15)
    sa, sb = C.clone_state(st), C.clone_state(st)
    fa, ra = P.step_learned(trained["R"], trained["Pl"], cn, en, sa, 3.0)
    fb, rb = P.step_learned(trained["R"], trained["Pl"], c2, e2, sb, 3.0)
    assert not fa and not fb
    assert all(torch_equal(sa[k], sb[k]) for k in sa)
    assert ra == pytest.approx(rb, rel=1e-5)   # FP32 per-block partial sums follow the chunking


def test_argument_errors(trained):
    P, C = trained["P"], trained["C"]
    st = _spun_up(trained, 16, steps=1)
    host = {k: v.cpu().numpy() for k, v in st.items()}
    with pytest.raises(P.IconError) as e:
        P.step_learned(trained["R"], trained["Pl"], trained["cn"], trained["en"], host, 3.0)
    assert e.value.code == P.ICON_ERR_ARG
    with pytest.raises(P.IconError) as e:   # the two networks swapped
        P.step_learned(trained["R"], trained["Pl"], trained["en"], trained["cn"], st, 3.0)
    assert e.value.code == P.ICON_ERR_ARG
    bare = P.MLP(trained["cn"].n_in, 64, trained["cn"].n_out, 1024)
    with pytest.raises(P.IconError) as e:   # no normalisation statistics
        P.step_learned(trained["R"], trained["Pl"], bare, trained["en"], st, 3.0)
    assert e.value.code == P.ICON_ERR_ARG
