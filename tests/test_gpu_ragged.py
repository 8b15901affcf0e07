"""GPU parity of the uneven-batch persistent solve (otlm_solve_ragged) against the FP64 oracle.

Every problem carries its own grid size, dictionary size, eps, grid and dictionary; each is
compared with the oracle run on that problem alone (trajectory parity, 1e-5 relative)."""
import numpy as np
import pytest

import oracle
import spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402

TOL32 = 1e-5


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def _run(problems, datafit, penalty, lam, alpha, iters, tol=0.0, tune=False):
    rb = api.ragged_batch(problems)
    w0 = np.concatenate([spectra.initial_weights(p["y"], p["D"]) for p in problems]).astype(np.float32)
    w = torch.tensor(w0, device="cuda")
    g = torch.zeros_like(rb.y)
    t = torch.empty_like(rb.y)
    B = len(problems)
    it = torch.empty(B, dtype=torch.int32, device="cuda")
    err = torch.empty(B, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    h = api.Handle(max(p["n"] for p in problems), max(p["k"] for p in problems), B, "fp32", datafit, penalty,
                   iters, tol, stream=torch.cuda.current_stream().cuda_stream)
    cta = h.tune_ragged(rb, lam, alpha, w, sample_every=3, iters=3) if tune else None
    h.solve_ragged(rb, lam, alpha, w, g, t, it, err, st)
    torch.cuda.synchronize()
    h.close()
    on = rb.off_n.cpu().numpy()
    okk = rb.off_k.cpu().numpy()
    out = []
    wn, tn, gn = w.cpu().numpy(), t.cpu().numpy(), g.cpu().numpy()
    for i, p in enumerate(problems):
        out.append(dict(w=wn[okk[i]:okk[i] + p["k"]], t=tn[on[i]:on[i] + p["n"]], g=gn[on[i]:on[i] + p["n"]]))
    return out, it.cpu().numpy(), err.cpu().numpy(), st.cpu().numpy(), cta, w0


def _oracle(p, datafit, penalty, lam, alpha, iters, tol=0.0):
    D = p["D"].astype(np.float64)
    y = p["y"].astype(np.float64)
    return oracle.solve_log(spectra.squared_cost(p["x"].astype(np.float64)), D, y, p["eps"], lam, alpha, datafit,
                            penalty, spectra.initial_weights(y, D), iters, tol=tol)


@pytest.mark.parametrize("datafit,penalty,lam,alpha", [("tv", "l1", 1.0, 1e-2), ("l2", "l2sq", 1.0, 1e-3),
                                                       ("kl", "l1", 1.0, 1e-2), ("poisson", "l2sq", 1.0, 1e-3)])
def test_ragged_trajectory_parity(datafit, penalty, lam, alpha):
    """Ten problems, n in [256, 700] (one and two rows per thread), k in [8, 60], own eps."""
    probs = spectra.ragged(41, 10, n_range=(256, 700), k_range=(8, 60))
    out, it, err, st, _, _ = _run(probs, datafit, penalty, lam, alpha, 25)
    assert np.all(it == 25) and np.all(st == api.MAX_ITER)
    for i, p in enumerate(probs):
        o = _oracle(p, datafit, penalty, lam, alpha, 25)
        assert rel_l1(out[i]["w"], o["w"]) <= TOL32, (i, p["n"], p["eps"], rel_l1(out[i]["w"], o["w"]))
        assert rel_l1(out[i]["t"], o["t"]) <= TOL32, (i, p["n"], p["eps"], rel_l1(out[i]["t"], o["t"]))


def test_ragged_mixed_sizes_including_n4096_and_edges():
    """n = 4096 (16 rows per thread), n = 2 and 3 (one thread), k = 1 and k = 128, extreme eps."""
    probs = spectra.ragged(42, 3, n_range=(900, 1500), k_range=(100, 128))
    big = spectra.ragged(43, 1, n_range=(4096, 4096), k_range=(128, 128))[0]
    tiny = [dict(x=np.array([0.0, 1.0], np.float32), D=np.array([[0.6], [0.4]], np.float32),
                 y=np.array([0.3, 0.5], np.float32), eps=0.5, n=2, k=1),
            dict(x=np.array([0.0, 0.5, 1.0], np.float32), D=np.array([[0.5, 0.1], [0.3, 0.3], [0.2, 0.6]], np.float32),
                 y=np.array([0.2, 0.5, 0.4], np.float32), eps=2e-3, n=3, k=2)]
    allp = probs + [big] + tiny
    out, it, err, st, _, _ = _run(allp, "tv", "l1", 1.0, 1e-2, 8)
    for i, p in enumerate(allp):
        o = _oracle(p, "tv", "l1", 1.0, 1e-2, 8)
        assert rel_l1(out[i]["w"], o["w"]) <= TOL32, (i, p["n"], rel_l1(out[i]["w"], o["w"]))
        assert rel_l1(out[i]["t"], o["t"]) <= TOL32, (i, p["n"], rel_l1(out[i]["t"], o["t"]))


def test_ragged_stopping_rule_and_tuner():
    """tol = 1e-5: each problem stops where the oracle stops, or one iteration apart when the
    oracle's violation at the deciding check lies within 5 % of tol.  The violation is built from
    |a_new/a_old - 1| ~ 1e-5, whose FP32 evaluation carries ~1e-7 absolute error: a few percent
    of tol.  The state is then compared at the GPU's own iteration count."""
    probs = spectra.ragged(44, 8, n_range=(256, 520), k_range=(8, 40))
    out, it, err, st, cta, w0 = _run(probs, "tv", "l1", 1.0, 1e-2, 2000, tol=1e-5, tune=True)
    assert cta in (128, 256, 512)
    assert np.all(st == api.CONVERGED) and np.all(err <= 1e-5)
    for i, p in enumerate(probs):
        o = _oracle(p, "tv", "l1", 1.0, 1e-2, 2000, tol=1e-5)
        gi = int(it[i])
        if gi != o["iters"]:
            e = o["err_hist"]
            assert abs(gi - o["iters"]) == 1 and abs(e[min(gi, o["iters"]) - 1] / 1e-5 - 1) < 5e-2
            o = _oracle(p, "tv", "l1", 1.0, 1e-2, gi)
        assert rel_l1(out[i]["w"], o["w"]) <= TOL32
        assert rel_l1(out[i]["t"], o["t"]) <= TOL32


def test_ragged_graph_replay_is_deterministic():
    probs = spectra.ragged(45, 6, n_range=(256, 400), k_range=(8, 20))
    rb = api.ragged_batch(probs)
    w0 = torch.tensor(np.concatenate([spectra.initial_weights(p["y"], p["D"]) for p in probs]).astype(np.float32),
                      device="cuda")
    h = api.Handle(400, 20, 6, "fp32", "tv", "l1", 12, 0.0, stream=torch.cuda.current_stream().cuda_stream)
    res = []
    for _ in range(3):
        w = w0.clone()
        t = torch.empty_like(rb.y)
        it = torch.empty(6, dtype=torch.int32, device="cuda")
        err = torch.empty(6, device="cuda")
        st = torch.empty(6, dtype=torch.int32, device="cuda")
        h.solve_ragged(rb, 1.0, 1e-2, w, None, t, it, err, st)
        torch.cuda.synchronize()
        res.append((w.cpu().numpy(), t.cpu().numpy()))
    h.close()
    for w_, t_ in res[1:]:
        np.testing.assert_array_equal(w_, res[0][0])
        np.testing.assert_array_equal(t_, res[0][1])


def _packed(problems, storage_order):
    """A RaggedBatch whose problems are stored in `storage_order` (problem indices stay 0..B-1):
    the offsets of problem p point at its place in that order, so they need not ascend."""
    B = len(problems)
    n = np.array([p["n"] for p in problems], np.int64)
    k = np.array([p["k"] for p in problems], np.int64)
    off_n, off_D, off_k = np.zeros(B, np.int64), np.zeros(B, np.int64), np.zeros(B, np.int64)
    on = oD = ok = 0
    for p in storage_order:
        off_n[p], off_D[p], off_k[p] = on, oD, ok
        on += n[p]
        oD += n[p] * k[p]
        ok += k[p]
    cat = lambda key: np.concatenate([np.asarray(problems[p][key], np.float32).ravel() for p in storage_order])  # noqa
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")  # noqa: E731
    w0 = np.concatenate([spectra.initial_weights(problems[p]["y"], problems[p]["D"]) for p in storage_order])
    return (api.RaggedBatch(B, t(n.astype(np.int32)), t(k.astype(np.int32)),
                            t(np.array([p["eps"] for p in problems], np.float32)), t(off_n), t(off_D), t(off_k),
                            t(cat("x")), t(cat("D")), t(cat("y"))), w0.astype(np.float32))


def test_ragged_offsets_in_any_order_and_out_of_range_offsets():
    """Problems packed in reverse order (offsets descending) give the same results as the ascending
    packing, through the tuner (whose temporary weights span sum k) and the solve; an offset range
    that leaves the packed arrays is refused before any work is queued."""
    probs = spectra.ragged(46, 7, n_range=(256, 600), k_range=(8, 40))
    B = len(probs)
    res = []
    for order in (list(range(B)), list(range(B))[::-1]):
        rb, w0 = _packed(probs, order)
        h = api.Handle(600, 40, B, "fp32", "tv", "l1", 10, 0.0, stream=torch.cuda.current_stream().cuda_stream)
        w = torch.tensor(w0, device="cuda")
        assert h.tune_ragged(rb, 1.0, 1e-2, w, sample_every=2, iters=2) in (128, 256, 512)
        t = torch.empty_like(rb.y)
        it = torch.empty(B, dtype=torch.int32, device="cuda")
        err = torch.empty(B, device="cuda")
        st = torch.empty(B, dtype=torch.int32, device="cuda")
        h.solve_ragged(rb, 1.0, 1e-2, w, None, t, it, err, st)
        torch.cuda.synchronize()
        on, ok = rb.off_n.cpu().numpy(), rb.off_k.cpu().numpy()
        wn, tn = w.cpu().numpy(), t.cpu().numpy()
        res.append([(wn[ok[p]:ok[p] + probs[p]["k"]], tn[on[p]:on[p] + probs[p]["n"]]) for p in range(B)])
        assert np.all(st.cpu().numpy() == api.MAX_ITER)
        if order[0] != 0:  # reversed packing: push one problem's weights past sum k
            bad = rb.off_k.clone()
            bad[0] = int(sum(p["k"] for p in probs)) - probs[0]["k"] + 1
            rb_bad = api.RaggedBatch(rb.batch, rb.n, rb.k, rb.eps, rb.off_n, rb.off_D, bad, rb.x, rb.D, rb.y)
            with pytest.raises(api.OTLMError):
                h.solve_ragged(rb_bad, 1.0, 1e-2, w, None, t, it, err, st)
            with pytest.raises(api.OTLMError):
                h.tune_ragged(rb_bad, 1.0, 1e-2, w, sample_every=2, iters=2)
        h.close()
    for p in range(B):
        np.testing.assert_array_equal(res[0][p][0], res[1][p][0])
        np.testing.assert_array_equal(res[0][p][1], res[1][p][1])


@pytest.mark.parametrize("cta,rows_log2", [(128, 3), (256, 3), (512, 1), (256, 5)])
def test_ragged_tile_shapes_from_the_table(cta, rows_log2):
    """Every size bucket forced to 2^rows_log2 rows per thread (raised where a CTA of `cta` threads
    needs more to cover n, and capped by what that CTA size compiles: 32 / 16 / 8 rows): each tile
    shape gives the oracle's trajectory at the 1e-5 bar (sizes span buckets 0-15)."""
    probs = spectra.ragged(47, 6, n_range=(256, 4096), k_range=(8, 64))
    B = len(probs)
    rb = api.ragged_batch(probs)
    w = torch.tensor(np.concatenate([spectra.initial_weights(p["y"], p["D"]) for p in probs]).astype(np.float32),
                     device="cuda")
    cap = {128: 5, 256: 4, 512: 3}[cta]
    h = api.Handle(4096, 64, B, "fp32", "tv", "l1", 6, 0.0, stream=torch.cuda.current_stream().cuda_stream,
                   ragged_cta=cta, ragged_rows_log2=[min(rows_log2, cap)] * 16)
    t = torch.empty_like(rb.y)
    it = torch.empty(B, dtype=torch.int32, device="cuda")
    err = torch.empty(B, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    h.solve_ragged(rb, 1.0, 1e-2, w, None, t, it, err, st)
    torch.cuda.synchronize()
    h.close()
    assert np.all(st.cpu().numpy() == api.MAX_ITER)
    on, ok = rb.off_n.cpu().numpy(), rb.off_k.cpu().numpy()
    wn, tn = w.cpu().numpy(), t.cpu().numpy()
    for i, p in enumerate(probs):
        o = _oracle(p, "tv", "l1", 1.0, 1e-2, 6)
        assert rel_l1(wn[ok[i]:ok[i] + p["k"]], o["w"]) <= TOL32, (i, p["n"])
        assert rel_l1(tn[on[i]:on[i] + p["n"]], o["t"]) <= TOL32, (i, p["n"])


def test_tuned_table_round_trips_through_otlm_create():
    """otlm_tune_ragged's table, given to a new handle through otlm_config, reproduces the tuned
    handle's results bit for bit."""
    probs = spectra.ragged(48, 40, n_range=(256, 2400), k_range=(8, 40))
    B = len(probs)
    rb = api.ragged_batch(probs)
    w0 = torch.tensor(np.concatenate([spectra.initial_weights(p["y"], p["D"]) for p in probs]).astype(np.float32),
                      device="cuda")
    res = []
    h = api.Handle(2400, 40, B, "fp32", "kl", "l1", 8, 0.0, stream=torch.cuda.current_stream().cuda_stream)
    cta, rows = h.tune_ragged(rb, 1.0, 1e-2, w0, sample_every=2, iters=2, with_rows=True)
    assert cta in (128, 256, 512) and all(0 <= r <= 5 for r in rows)
    h2 = api.Handle(2400, 40, B, "fp32", "kl", "l1", 8, 0.0, stream=torch.cuda.current_stream().cuda_stream,
                    ragged_cta=cta, ragged_rows_log2=rows)
    for hh in (h, h2):
        w = w0.clone()
        t = torch.empty_like(rb.y)
        it = torch.empty(B, dtype=torch.int32, device="cuda")
        err = torch.empty(B, device="cuda")
        st = torch.empty(B, dtype=torch.int32, device="cuda")
        hh.solve_ragged(rb, 1.0, 1e-2, w, None, t, it, err, st)
        torch.cuda.synchronize()
        res.append((w.cpu().numpy(), t.cpu().numpy()))
        hh.close()
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])
