"""Host-side logic that needs no GPU: the source sharding and gradient sum of the multi-rank
path (two gloo ranks on CPU), the chunking of the autograd objective, the outer loop's control
flow and checkpoints, and the on-disk autotune cache."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_partitions_every_count():
    from paper_2410_18429_gb300.parallel_sum import shard
    for n in (0, 1, 7, 128, 384):
        for world in (1, 2, 3, 8):
            parts = [shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (b0, e0), (b1, e1) in zip(parts, parts[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    from paper_2410_18429_gb300.parallel_sum import allreduce_gradient, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank owns a shard of 10 systems; its gradient is the sum of per-system terms
    b, e = shard(10, rank, world)
    # two frequency groups on grids of different shapes
    per_system = [torch.arange(12, dtype=torch.float64).reshape(2, 2, 3) * (s + 1) for s in range(10)]
    per_system_b = [torch.arange(20, dtype=torch.float64).reshape(4, 5) - s for s in range(10)]
    g = [sum(per_system[b:e], torch.zeros(2, 2, 3, dtype=torch.float64)),
         sum(per_system_b[b:e], torch.zeros(4, 5, dtype=torch.float64))]
    f = torch.tensor([float(sum(s + 1 for s in range(b, e)))], dtype=torch.float64)
    out = allreduce_gradient(g, f)
    assert out[0] is g and out[1] is f                       # summed in place
    torch.save({"g": g[0], "g_b": g[1], "f": f}, os.path.join(out_dir, f"r{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


def test_gradient_allreduce_two_gloo_ranks(tmp_path):
    """World size 2 on CPU: the summed gradient equals the gradient of all systems on one rank."""
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    want_g = torch.arange(12, dtype=torch.float64).reshape(2, 2, 3) * sum(range(1, 11))
    want_b = torch.arange(20, dtype=torch.float64).reshape(4, 5) * 10 - sum(range(10))
    for r in range(2):
        got = torch.load(os.path.join(tmp_path, f"r{r}.pt"))
        assert torch.equal(got["g"], want_g) and torch.equal(got["g_b"], want_b)
        assert got["f"].item() == 55.0


def _sharded_eval_main(rank, world, port, out_dir):
    """One rank of a sharded WRI evaluation: its share of the systems (parallel_sum.shard) is
    evaluated (the CPU oracle stands in for the GPU library here), then the one exchange step."""
    import numpy as np
    import torch.distributed as dist

    import oracle as O
    from paper_2410_18429_gb300.parallel_sum import allreduce_gradient, shard
    from wri_cases import case
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    G = case(nphys=(7, 6, 5), npml=3, nsys=5, seed=21, freq=14.0)
    b, e = shard(G.nsys, rank, world)
    off = G.rec_off[b:e + 1]
    _, _, f, g = O.evaluate(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src[b:e], off - off[0],
                            G.rec_idx[off[0]:off[-1]], G.d[off[0]:off[-1]], G.lam)
    gt = [torch.as_tensor(np.asarray(g, dtype=np.float64).reshape(G.spec.shape))]
    ft = torch.tensor([f], dtype=torch.float64)
    allreduce_gradient(gt, ft)
    torch.save({"g": gt[0], "f": ft, "share": (b, e)}, os.path.join(out_dir, f"e{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_wri_evaluation_two_gloo_ranks(tmp_path):
    """World size 2 on CPU: 5 systems split 3 + 2 over the ranks, each rank's WRI objective and gradient
    of its share, one all-reduce: every rank holds the f and g of all 5 systems on one rank."""
    import torch.multiprocessing as mp

    import oracle as O
    from wri_cases import case
    port = _free_port()
    mp.start_processes(_sharded_eval_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    G = case(nphys=(7, 6, 5), npml=3, nsys=5, seed=21, freq=14.0)
    _, _, f, g = O.evaluate(G.spec.shape, G.spec.h, G.omega, G.m, G.spec.npml, G.v_max, G.src, G.rec_off, G.rec_idx,
                            G.d, G.lam)
    shares = []
    for r in range(2):
        got = torch.load(os.path.join(tmp_path, f"e{r}.pt"))
        shares.append(tuple(got["share"]))
        assert abs(got["f"].item() - f) <= 1e-12 * abs(f)
        assert torch.allclose(got["g"].reshape(-1), torch.as_tensor(g), rtol=0, atol=1e-12 * float(np.abs(g).max()))
    assert shares == [(0, 3), (3, 5)]


def test_allreduce_is_identity_without_process_group():
    from paper_2410_18429_gb300.parallel_sum import allreduce_gradient
    g = [torch.ones(3, dtype=torch.float64)]
    f = torch.tensor([2.0], dtype=torch.float64)
    allreduce_gradient(g, f)
    assert torch.equal(g[0], torch.ones(3, dtype=torch.float64)) and f.item() == 2.0


def test_objective_chunks_cover_systems():
    from paper_2410_18429_gb300.objective import chunks
    assert chunks(0, 4) == []
    assert chunks(5, 2) == [(0, 2), (2, 4), (4, 5)]
    assert chunks(3, 1 << 30) == [(0, 3)]
    for n in range(0, 20):
        for k in (1, 3, 7, 50):
            c = chunks(n, k)
            assert sum(e - b for b, e in c) == n and all(0 < e - b <= k for b, e in c)
    with pytest.raises(ValueError):
        chunks(3, 0)


def test_workload_shards_differ_only_in_weights_and_data():
    """Rank r's shot record shares the geometry and model of rank 0 but not its weights or traces."""
    import synth
    a = synth.workload_c4(nsrc=4, freqs=((3.0, 16),), nrec=8, shard=0)[0]
    b = synth.workload_c4(nsrc=4, freqs=((3.0, 16),), nrec=8, shard=1)[0]
    assert np.array_equal(a.src, b.src) and np.array_equal(a.rec_idx, b.rec_idx) and np.array_equal(a.m, b.m)
    assert not np.allclose(a.alpha, b.alpha) and not np.allclose(a.d, b.d)


def test_lbfgs_product_matches_oracle_two_loop():
    """The product's l-BFGS product (torch) equals the oracle's two-loop recursion (numpy)."""
    from oracle.awri_oracle import two_loop
    from paper_2410_18429_gb300.awri import LBFGS
    r = np.random.Generator(np.random.PCG64(41))
    n = 15
    Q = r.standard_normal((n, n))
    Q = Q @ Q.T + n * np.eye(n)
    lb = LBFGS(memory=3)
    S, Y = [], []
    for _ in range(5):
        s = r.standard_normal(n)
        y = Q @ s
        assert lb.update(torch.as_tensor(s), torch.as_tensor(y))
        S.append(s)
        Y.append(y)
    g = r.standard_normal(n)
    got = lb.apply(torch.as_tensor(g)).numpy()
    assert np.allclose(got, two_loop(g, S[-3:], Y[-3:]), rtol=1e-12, atol=1e-14)
    assert not lb.update(torch.as_tensor(S[0]), torch.as_tensor(-Y[0]))   # s.y < 0: refused


def test_awri_product_loop_matches_oracle_loop():
    """The product's Algorithm 2 control flow (tolerance halving, acceptance, l-BFGS pairs) gives
    the oracle's iterates on the same objective, including halvings."""
    from oracle.awri_oracle import awri as awri_oracle
    from paper_2410_18429_gb300.awri import awri
    r = np.random.Generator(np.random.PCG64(7))
    n = 10
    U, _ = np.linalg.qr(r.standard_normal((n, n)))
    Q = U @ np.diag(np.linspace(1.0, 30.0, n)) @ U.T
    m_star = r.uniform(1.0, 2.0, n)
    c = r.standard_normal(n)

    def f_np(m, eps):
        # exact objective, gradient with an eps-sized error (as from loosely solved systems)
        e = m - m_star
        return 0.5 * e @ Q @ e, Q @ e + 200.0 * eps * c

    def f_torch(m, eps):
        f, g = f_np(m.numpy(), eps)
        return float(f), torch.as_tensor(g)

    m0 = np.full(n, 1.5)
    mo, fo, so, ho = awri_oracle(m0, f_np, 0.2, 8, first_step=0.3, eps_min=1e-6)
    res = awri(torch.as_tensor(m0), f_torch, 0.2, 8, first_step=0.3, eps_min=1e-6)
    assert res.status == so
    assert [h["eps"] for h in res.history] == [h["eps"] for h in ho]
    assert any(h["eps"] < 0.2 for h in ho)           # the case exercises the halving
    assert np.allclose(res.m.numpy(), mo, rtol=1e-12, atol=1e-14)
    assert abs(res.f - fo) <= 1e-12 * abs(fo)


def test_objective_chunk_slices_geometry_and_data():
    """A chunk [b, e) of a group keeps exactly its systems' sources, receiver lists (CSR offsets
    rebased to 0), data entries and known weights, and takes the given model and wavefields."""
    from dataclasses import replace

    from paper_2410_18429_gb300.objective import _sub
    from paper_2410_18429_gb300.wri import GroupSpec
    rec_off = np.array([0, 3, 5, 9, 10], np.int32)
    rec_idx = np.arange(10, dtype=np.int32) * 7
    d = torch.arange(10, dtype=torch.float32).to(torch.complex64)
    alpha = torch.arange(8, dtype=torch.float64).reshape(4, 2)
    g = GroupSpec(8, 6, 5, 1, 10.0, 30.0, 2000.0, None, np.array([11, 22, 33, 44], np.int64), rec_off, rec_idx, d,
                  0.01, None, alpha)
    m = torch.zeros(5, 6, 8)
    u = torch.zeros(2, 240, dtype=torch.complex64)
    s = _sub(g, 1, 3, m, u)
    assert s.src.tolist() == [22, 33] and s.nsys == 2
    assert s.rec_off.tolist() == [0, 2, 6] and s.rec_off.dtype == np.int32
    assert s.rec_idx.tolist() == [21, 28, 35, 42, 49, 56]
    assert s.d.real.tolist() == [3, 4, 5, 6, 7, 8]
    assert s.alpha.tolist() == [[2.0, 3.0], [4.0, 5.0]]
    assert s.m is m and s.u is u and s.u64 is None and (s.nx, s.ny, s.nz, s.lam) == (8, 6, 5, 0.01)
    s2 = _sub(replace(g, alpha=None), 0, 4, m, u)
    assert s2.alpha is None and s2.rec_off.tolist() == rec_off.tolist()



def test_awri_checkpoint_and_resume_continue_exactly(tmp_path):
    """Eight iterations straight equal three iterations checkpointed to disk, the state loaded
    back, and the loop continued to eight: the same iterates, objective values, tolerances
    (halvings included) and evaluation count, bit for bit."""
    from paper_2410_18429_gb300.awri import awri, load_state
    r = np.random.Generator(np.random.PCG64(7))
    n = 10
    U, _ = np.linalg.qr(r.standard_normal((n, n)))
    Q = torch.as_tensor(U @ np.diag(np.linspace(1.0, 30.0, n)) @ U.T)
    m_star = torch.as_tensor(r.uniform(1.0, 2.0, n))
    c = torch.as_tensor(r.standard_normal(n))
    calls = []

    def evaluate(m, eps):
        calls.append(eps)
        e = m - m_star
        return float(0.5 * e @ Q @ e), Q @ e + 200.0 * eps * c

    m0 = torch.full((n,), 1.5, dtype=torch.float64)
    full = awri(m0, evaluate, 0.2, 8, first_step=0.3, eps_min=1e-6)
    n_full = len(calls)
    assert any(h["eps"] < 0.2 for h in full.history[3:])     # halvings after the checkpoint too
    calls.clear()
    path = str(tmp_path / "awri_state.pt")
    part = awri(m0, evaluate, 0.2, 3, first_step=0.3, eps_min=1e-6, checkpoint=path)
    st = load_state(path)
    assert st.iteration == 3 and len(st.s) == len(part.state.s) and st.eps == part.state.eps
    rest = awri(None, evaluate, 0.2, 8, first_step=0.3, eps_min=1e-6, state=st)
    assert len(calls) == n_full and rest.evaluations == full.evaluations
    assert torch.equal(rest.m, full.m) and rest.f == full.f and rest.status == full.status
    assert rest.history == full.history
    with pytest.raises(ValueError):
        awri(None, evaluate, 0.2, 8)


def test_autotune_disk_cache(tmp_path, monkeypatch):
    """The on-disk autotune cache: a miss runs the library's trials and stores the choice, a hit
    for the same GPU, build, options and batch reuses it without trials, and a change in any of
    them (or an unreadable file) runs the trials again.  The library is a fake that records its
    calls (no GPU); the key logic and the file handling are the product's."""
    from paper_2410_18429_gb300 import wri

    class FakeLib:
        def __init__(self):
            self.calls = 0
            self.ver = b"libwri fake src 000"

        def wri_workspace_size(self, arr, n, opts):
            return 1024

        def wri_autotune(self, arr, n, opts_ref, trial_iters, ws, nbytes, stream):
            self.calls += 1
            opts_ref._obj.kernel, opts_ref._obj.order = 2 + 18, 5
            return wri.OK

        def wri_version(self):
            return self.ver

        def wri_strerror(self, code):
            return b"fake"

    fake = FakeLib()
    monkeypatch.setattr(wri, "lib", fake)
    monkeypatch.setattr(wri, "_stream", lambda stream=None: None)
    monkeypatch.delenv("WRI_TUNE_CACHE", raising=False)

    class Ptr:
        """A device-pointer holder (not a tensor): the fake library never dereferences it."""
        device = torch.device("cpu")

        def data_ptr(self):
            return 0x1000

    def group(nsys):
        return wri.GroupSpec(6, 5, 4, 1, 10.0, 30.0, 2000.0, Ptr(), np.arange(nsys, dtype=np.int64),
                             np.arange(nsys + 1, dtype=np.int32), np.arange(nsys, dtype=np.int32) + 50,
                             Ptr(), 0.01, Ptr())

    opts = wri.make_opts(tol=1e-3, max_iter=100)
    path = str(tmp_path / "tune.json")
    out = wri.autotune([group(3)], opts, cache=path)
    assert (fake.calls, out.kernel, out.order) == (1, 20, 5) and (opts.kernel, opts.order) == (0, 0)
    out = wri.autotune([group(3)], opts, cache=path)                     # hit: no trials
    assert (fake.calls, out.kernel, out.order) == (1, 20, 5)
    monkeypatch.setenv("WRI_TUNE_CACHE", path)                           # the same file through the variable
    assert wri.autotune([group(3)], opts).kernel == 20 and fake.calls == 1
    wri.autotune([group(4)], opts)                                       # another batch shape
    assert fake.calls == 2
    wri.autotune([group(3)], wri.make_opts(tol=1e-3, max_iter=100, dtype=wri.C128))   # other options
    assert fake.calls == 3
    fake.ver = b"libwri fake src 111"                                    # a rebuilt library
    wri.autotune([group(3)], opts)
    assert fake.calls == 4
    with open(path) as fh:
        assert len(json.load(fh)) == 4
    with open(path, "w") as fh:
        fh.write("{not json")
    wri.autotune([group(3)], opts)                                       # unreadable file: trials, rewritten
    assert fake.calls == 5
    with open(path) as fh:
        assert len(json.load(fh)) == 1
    monkeypatch.delenv("WRI_TUNE_CACHE")
    wri.autotune([group(3)], opts)                                       # no cache: always trials
    wri.autotune([group(3)], opts)
    assert fake.calls == 7
