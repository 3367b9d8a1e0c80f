"""The request server: results alone equal results in a mix of concurrent
requests (bit for bit: every solve uses only its own scratch and fixed-order
reductions), every result meets tol on the true residual (re-formed by the
CPU oracle), and admission never exceeds the byte budget."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import residual_limit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spx():
    from paper_2103_10116_gb300 import spx as s
    s.load()
    return s


@pytest.fixture(scope="module")
def ctx(spx):
    c = spx.spx_ctx_create(0)
    yield c
    spx.spx_ctx_destroy(c)


def _requests(large=False):
    reqs = []
    if large:  # above the batch lanes' size limit: solved on a slot of its own
        rp, col, val = synth.laplace3d_7pt(32)
        reqs.append((rp, col, val, synth.uniform_vector(32**3, seed=99), "cg"))
    for k, m in enumerate((10, 14, 18, 22, 26)):
        rp, col, val = synth.laplace3d_7pt(m)
        b = synth.uniform_vector(m**3, seed=100 + k)
        reqs.append((rp, col, val, b, "cg"))
    for k, n in enumerate((1000, 4000, 9000, 20000)):
        rp, col, val = synth.diagdom_random(n, seed=200 + k)
        b = synth.uniform_vector(n, seed=300 + k)
        reqs.append((rp, col, val, b, "bicgstab" if k < 3 else "cgs"))
    return reqs


@pytest.mark.parametrize("batch_rows,cluster_rows", [(None, None), (65536, None), (0, None), (0, 0)])
def test_alone_equals_mix(spx, ctx, batch_rows, cluster_rows):
    """batch_rows None (the default, 24576): small requests go through the
    batch lanes, the large one (32^3 rows) through a slot; 65536: the large
    one is batched too, its gathered vector in global memory; 0: every
    request on a slot of its own (the short-row ones up to 65536 rows as
    one-cluster solves, the default; with cluster_rows 0 on the general path)."""
    from paper_2103_10116_gb300.serving import Server
    reqs = _requests(large=True)
    srv = Server(ctx, 0, max_slots=4, batch_rows=batch_rows)
    eff = spx.spx_server_set_batching(srv.h, -1)
    assert eff == (24576 if batch_rows is None else batch_rows)
    if cluster_rows is not None:
        spx.spx_server_set_cluster_rows(srv.h, cluster_rows)
    cl_rows = spx.spx_server_set_cluster_rows(srv.h, -1)
    assert cl_rows == (65536 if cluster_rows is None else cluster_rows)
    try:
        alone = {}
        for i, (rp, col, val, b, solver) in enumerate(reqs):
            rid = srv.submit(rp, col, val, b, solver=solver, tol=1e-8)
            srv.drain()
            alone[i] = srv.results[rid]
        mix_ids = {}
        order = list(range(len(reqs))) * 3
        np.random.default_rng(1).shuffle(order)
        for i in order:
            rp, col, val, b, solver = reqs[i]
            mix_ids.setdefault(i, []).append(srv.submit(rp, col, val, b, solver=solver, tol=1e-8))
        srv.drain()
        # routes: batch lanes up to the batch limit; above it (or with the lanes off)
        # short-row operators of at most cl_rows rows solve on one cluster, the rest on the general path
        for i, (rp, col, val, b, solver) in enumerate(reqs):
            n = rp.shape[0] - 1
            short = col.shape[0] <= 8 * n
            want = "batch" if n <= eff else ("cluster" if short and n <= cl_rows else "slot")
            assert alone[i]["route"] == want, (i, n, alone[i]["route"])
        for i, (rp, col, val, b, solver) in enumerate(reqs):
            ra = alone[i]
            assert ra["error"] == 0 and ra["info"].status == spx.SPX_CONVERGED, ra
            r = b - oracle.spmv_csr(rp, col, val, ra["x"])
            assert np.linalg.norm(r) / np.linalg.norm(b) <= residual_limit(rp, col, val, b, ra["x"], 1e-8)
            for rid in mix_ids[i]:
                rm = srv.results[rid]
                assert rm["error"] == 0 and rm["info"].status == spx.SPX_CONVERGED
                assert np.array_equal(rm["x"], ra["x"]), i
                assert rm["info"].iterations == ra["info"].iterations
        # the mix really overlapped: some request was admitted before another finished
        res = [srv.results[r] for ids in mix_ids.values() for r in ids]
        res.sort(key=lambda r: r["admit_ms"])
        assert any(res[k + 1]["admit_ms"] < res[k]["done_ms"] for k in range(len(res) - 1))
    finally:
        srv.close()


def test_admission_respects_budget(spx, ctx):
    from paper_2103_10116_gb300.serving import Server
    reqs = _requests()
    budget = 12 * 2**20  # ~12 MB: only a few of the small requests fit at once
    srv = Server(ctx, budget, max_slots=8)
    try:
        big = synth.laplace3d_7pt(60)
        with pytest.raises(spx.SpxError) as ei:
            srv.submit(big[0], big[1], big[2], np.ones(60**3))
        assert ei.value.status == spx.SPX_ERR_TOO_LARGE
        srv.live.clear()
        ids = []
        for i in range(3):
            for rp, col, val, b, solver in reqs[:4]:
                ids.append(srv.submit(rp, col, val, b, solver=solver))
        peak = 0
        while srv.live:
            q, running, used = spx.spx_server_pending(srv.h)
            peak = max(peak, used)
            assert used <= budget
            srv.poll(wait_ms=5)
        assert peak > 0
        assert all(srv.results[i]["info"].status == spx.SPX_CONVERGED for i in ids)
    finally:
        srv.close()


def test_invalid_operator_in_batch_is_rejected_alone(spx, ctx):
    """A batched request with a column out of range fails with SPX_ERR_INVALID
    and does not disturb the requests batched with it."""
    from paper_2103_10116_gb300.serving import Server
    reqs = _requests()[:3]
    rp, col, val = synth.laplace3d_7pt(8)
    bad = col.copy()
    bad[5] = 8**3 + 3
    srv = Server(ctx, 0, max_slots=2)
    try:
        ids = [srv.submit(rp_, col_, val_, b_, solver=s_) for rp_, col_, val_, b_, s_ in reqs]
        bad_id = srv.submit(rp, bad, val, np.ones(8**3), solver="cg")
        srv.drain()
        assert srv.results[bad_id]["error"] == spx.SPX_ERR_INVALID
        for i in ids:
            assert srv.results[i]["error"] == 0 and srv.results[i]["info"].status == spx.SPX_CONVERGED
    finally:
        srv.close()


def test_preconditioned_requests_alone_equal_mix(spx, ctx):
    """Jacobi and block-Jacobi requests (a slot each: the batch lanes do not
    precondition) converge and give the same result alone and in a mix."""
    from paper_2103_10116_gb300.serving import Server
    rp, col, val = synth.laplace3d_7pt(14)
    b = synth.uniform_vector(14**3, seed=7)
    rp2, col2, val2 = synth.diagdom_random(6000, seed=8)
    b2 = synth.uniform_vector(6000, seed=9)
    codes = [(rp, col, val, b, spx.SPX_CG | spx.SPX_PRECOND_JACOBI),
             (rp, col, val, b, spx.SPX_CG | spx.SPX_PRECOND_BLOCK(8)),
             (rp2, col2, val2, b2, spx.SPX_BICGSTAB | spx.SPX_PRECOND_BLOCK(4) | spx.SPX_PRECOND_BLOCK_ADAPTIVE),
             (rp2, col2, val2, b2, spx.SPX_GMRES | spx.SPX_PRECOND_BLOCK(16))]
    srv = Server(ctx, 0, max_slots=4)
    try:
        alone = []
        for rpx, colx, valx, bx, code in codes:
            rid = srv.submit(rpx, colx, valx, bx, solver=code, tol=1e-8)
            srv.drain()
            alone.append(srv.results[rid])
        ids = [srv.submit(c[0], c[1], c[2], c[3], solver=c[4], tol=1e-8) for c in codes * 2]
        srv.drain()
        for k, (rpx, colx, valx, bx, code) in enumerate(codes):
            ra = alone[k]
            assert ra["error"] == 0 and ra["info"].status == spx.SPX_CONVERGED, ra
            r = bx - oracle.spmv_csr(rpx, colx, valx, ra["x"])
            assert np.linalg.norm(r) / np.linalg.norm(bx) <= residual_limit(rpx, colx, valx, bx, ra["x"], 1e-8)
            for rid in (ids[k], ids[k + len(codes)]):
                assert np.array_equal(srv.results[rid]["x"], ra["x"])
    finally:
        srv.close()


def test_resident_matrix_requests(spx, ctx):
    """Requests on resident matrix handles: nothing of the operator is uploaded
    (set-up time 0), a handle serves several requests (one at a time, the
    others overlapping with requests on other handles), every result meets
    tol on the oracle-formed residual and equals the same request alone, bit
    for bit; the phase times are reported."""
    from paper_2103_10116_gb300.serving import Server
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
    mats = [synth.laplace3d_7pt(24), synth.laplace3d_7pt(30)]
    handles = [spx.spx_matrix_create(ctx, "csr", t(rp), t(col), t(val), flags=spx.SPX_MIXED_SHADOW)
               for rp, col, val in mats]
    torch.cuda.synchronize()
    srv = Server(ctx, 0, max_slots=4, batch_rows=0)
    try:
        bs = [[synth.uniform_vector(rp.shape[0] - 1, seed=400 + 10 * h + k) for k in range(3)]
              for h, (rp, _, _) in enumerate(mats)]
        alone = {}
        for h in range(2):
            for k in range(3):
                rid = srv.submit_matrix(handles[h], bs[h][k], solver="cg", tol=1e-8)
                srv.drain()
                alone[(h, k)] = srv.results[rid]
        ids = {}
        for k in range(3):
            for h in range(2):
                ids[(h, k)] = srv.submit_matrix(handles[h], bs[h][k], solver="cg", tol=1e-8)
        srv.drain()
        for (h, k), rid in ids.items():
            rm, ra = srv.results[rid], alone[(h, k)]
            rp, col, val = mats[h]
            b = bs[h][k]
            assert rm["error"] == 0 and rm["info"].status == spx.SPX_CONVERGED, rm
            r = b - oracle.spmv_csr(rp, col, val, rm["x"])
            assert np.linalg.norm(r) / np.linalg.norm(b) <= residual_limit(rp, col, val, b, rm["x"], 1e-8)
            assert np.array_equal(rm["x"], ra["x"])
            assert rm["setup_ms"] == 0.0 or rm["setup_ms"] < 1.0  # no operator to build
            assert rm["solve_ms"] > 0 and not rm["batched"]
        # requests on one handle never overlapped
        for h in range(2):
            spans = sorted((srv.results[ids[(h, k)]]["admit_ms"], srv.results[ids[(h, k)]]["done_ms"])
                           for k in range(3))
            assert all(spans[i][1] <= spans[i + 1][0] for i in range(2)), spans
    finally:
        srv.close()
        for A in handles:
            spx.spx_matrix_destroy(A)


def test_phase_times_of_uploaded_requests(spx, ctx):
    from paper_2103_10116_gb300.serving import Server
    srv = Server(ctx, 0, max_slots=2, batch_rows=24576)
    try:
        rp, col, val = synth.laplace3d_7pt(34)       # a slot request
        rps, cols, vals = synth.laplace3d_7pt(12)    # a batched request
        b, bsm = synth.uniform_vector(34**3, seed=7), synth.uniform_vector(12**3, seed=8)
        r1 = srv.submit(rp, col, val, b, solver="cg", tol=1e-8)
        r2 = srv.submit(rps, cols, vals, bsm, solver="cg", tol=1e-8)
        srv.drain()
        big, small = srv.results[r1], srv.results[r2]
        assert not big["batched"] and small["batched"]
        for r in (big, small):
            assert r["error"] == 0 and r["info"].status == spx.SPX_CONVERGED
            phases = r["upload_ms"] + r["setup_ms"] + r["solve_ms"] + r["download_ms"]
            assert min(r["upload_ms"], r["setup_ms"], r["solve_ms"], r["download_ms"]) >= 0
            assert phases <= r["done_ms"] - r["admit_ms"] + 1e-6
            assert r["solve_ms"] > 0
    finally:
        srv.close()


@pytest.mark.parametrize("which", ["stencil29", "random4645", "stencil12"])
def test_single_request_batches(spx, ctx, which):
    """A batch lane solving one request alone, at sizes the trace produced when a
    launch was once refused (a shared-memory carve-out hint that did not fit):
    every request completes without error and meets tol."""
    from paper_2103_10116_gb300.serving import Server
    if which.startswith("stencil"):
        m = int(which[7:])
        rp, col, val = synth.laplace3d_7pt(m)
        solver = "cg"
    else:
        rp, col, val = synth.diagdom_random(int(which[6:]), seed=3)
        solver = "bicgstab"
    b = synth.uniform_vector(rp.shape[0] - 1, seed=11)
    srv = Server(ctx, 0, max_slots=2)
    try:
        for _ in range(2):
            rid = srv.submit(rp, col, val, b, solver=solver, tol=1e-8)
            srv.drain()
            r = srv.results[rid]
            assert r["error"] == 0 and r["batched"] and r["info"].status == spx.SPX_CONVERGED, r
            res = b - oracle.spmv_csr(rp, col, val, r["x"])
            assert np.linalg.norm(res) / np.linalg.norm(b) <= residual_limit(rp, col, val, b, r["x"], 1e-8)
    finally:
        srv.close()


def test_concurrent_lanes_of_different_sizes(spx, ctx):
    """Many small requests of every batch size class at once: the four batch
    lanes launch the batched kernel concurrently with different shared-memory
    sizes, and no launch may be refused (the shared-memory opt-in only grows)."""
    from paper_2103_10116_gb300.serving import Server
    rng = np.random.default_rng(8)
    sizes = rng.integers(800, 24000, size=160)
    mats = {}
    srv = Server(ctx, 0, max_slots=2, keep_x=False)
    try:
        ids = []
        for k, n in enumerate(sizes):
            n = int(n)
            if n not in mats:
                mats[n] = synth.diagdom_random(n, seed=n % 97)
            rp, col, val = mats[n]
            ids.append(srv.submit(rp, col, val, synth.uniform_vector(n, seed=k), solver="bicgstab", tol=1e-8))
        srv.drain()
        for rid in ids:
            r = srv.results[rid]
            assert r["error"] == 0 and r["info"].status == spx.SPX_CONVERGED, r
    finally:
        srv.close()


def test_cluster_route_setting_and_flag(spx, ctx):
    """spx_server_set_cluster_rows(0) keeps short-row slot requests on the
    general path; SPX_SOLVE_ONE_CLUSTER in a request's solver code sends it to
    the cluster route whatever its rows; both routes meet tol."""
    from paper_2103_10116_gb300.serving import Server
    rp, col, val = synth.laplace3d_7pt(32)
    b = synth.uniform_vector(32**3, seed=5)
    rpd, cold, vald = synth.diagdom_random(30000, seed=6)
    bd = synth.uniform_vector(30000, seed=7)
    srv = Server(ctx, 0, max_slots=2)
    try:
        assert spx.spx_server_set_cluster_rows(srv.h, -1) == 65536  # the default
        assert spx.spx_server_set_slot_sms(srv.h, -2) == 0  # the default: whole-device grids
        assert spx.spx_server_set_slot_sms(srv.h, -1) == -1  # grid share by row length from here on
        a = srv.submit(rp, col, val, b, solver="cg", tol=1e-8)
        d = srv.submit(rpd, cold, vald, bd, solver="bicgstab", tol=1e-8)
        f = srv.submit(rpd, cold, vald, bd, solver=spx.SPX_BICGSTAB | spx.SPX_SOLVE_ONE_CLUSTER, tol=1e-8)
        srv.drain()
        assert spx.spx_server_set_cluster_rows(srv.h, 0) == 0
        g = srv.submit(rp, col, val, b, solver="cg", tol=1e-8)
        srv.drain()
        routes = [srv.results[i]["route"] for i in (a, d, f, g)]
        assert routes == ["cluster", "slot", "cluster", "slot"], routes
        for i, (rp_, col_, val_, b_) in ((a, (rp, col, val, b)), (d, (rpd, cold, vald, bd)),
                                         (f, (rpd, cold, vald, bd)), (g, (rp, col, val, b))):
            r = srv.results[i]
            assert r["error"] == 0 and r["info"].status == spx.SPX_CONVERGED, r
            x = r["x"]
            rel = np.linalg.norm(b_ - oracle.spmv_csr(rp_, col_, val_, x)) / np.linalg.norm(b_)
            assert rel <= residual_limit(rp_, col_, val_, b_, x, 1e-8), (i, rel)
    finally:
        srv.close()
