"""Batched discs and the asynchronous (graph-capturable) step, on the GPU.

Batched discs: several independent discs of uneven grid and bin counts,
integrated side by side through cudisc_coag_batch_step; every disc is
checked against the oracle replaying that disc's own accepted step
sequence (tolerances as in test_gpu_mixed: 1e-5 relative with the paper's
absolute tolerance 1e-10 S as the floor; FP64 1e-10).  The asynchronous
step is captured in a CUDA graph, replayed, and compared with the
synchronous call on the same input.
"""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def small_batch():
    """Four discs: cell counts 24..600, 17..72 bins, different alpha and v_frag."""
    return [
        synth.make_disc(3, 8, 17, 1e-5, 0.1, 10.0, 20.0, 100.0, alpha=1e-2, v_frag=300.0, seed=31),
        synth.make_disc(20, 30, 40, 1e-5, 1.0, 5.0, 100.0, 300.0, alpha=1e-3, v_frag=100.0, seed=32),
        synth.make_disc(6, 10, 72, 1e-5, 10.0, 5.0, 50.0, 300.0, alpha=1e-4, v_frag=1000.0, seed=33),
        synth.make_disc(12, 16, 33, 1e-5, 1.0, 10.0, 100.0, 200.0, alpha=3e-3, v_frag=500.0, seed=34),
    ]


def check_rel(out, ref, S, rel, atol_rel=1e-10):
    r = np.abs(out - ref) / (rel * np.abs(ref) + atol_rel * S[:, None])
    assert r.max() <= 1.0, r.max()


@pytest.mark.parametrize("precision,rel", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_batched_discs_match_oracle(coag_mod, oracle_mod, precision, rel):
    discs = small_batch()
    b = coag_mod.Batch(discs, precision)
    recs = [b.disc(i).set_records(4000) for i in range(len(b))]
    ys = [b.disc(i).state(d.rho0) for i, d in enumerate(discs)]
    stats = b.step(ys, discs[0].t_span)
    for i, d in enumerate(discs):
        st = stats[i]
        assert st["worst_status"] == 0 and st["n_failed"] == 0
        assert st["mass_err_max"] < 1e-9
        n = recs[i]["n"].cpu().numpy()
        assert st["accepted"] == n.sum()
        cells = np.unique(np.linspace(0, d.n_cells - 1, 6).astype(int))
        want = oracle_mod.Oracle(d.subset(cells)).replay(d.rho0[cells], recs[i]["dt"].cpu().numpy()[cells],
                                                         n[cells])
        check_rel(ys[i].cpu().numpy()[cells], want, d.rho0[cells].sum(1), rel)
    b.close()


def test_batch_shares_the_sms(coag_mod):
    """Every disc's persistent grid fits in its share, the shares in the GPU."""
    discs = small_batch()
    b = coag_mod.Batch(discs, "mixed")
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    used = 0
    for i in range(len(b)):
        P, groups = b.disc(i).mixed_cluster()
        assert P >= 1 and groups >= 1
        used += P * groups
    assert used <= n_sm
    b.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_step_in_one_cuda_graph(coag_mod, precision):
    """All discs of a batch captured as one graph (each disc forked from the
    capturing stream and joined back), replayed twice: bitwise the
    synchronous batch step, the same accepted counts."""
    discs = small_batch()
    b = coag_mod.Batch(discs, precision)
    init = [b.disc(i).state(d.rho0) for i, d in enumerate(discs)]
    refs = [x.clone() for x in init]
    stats = b.step(refs, discs[0].t_span)
    assert all(st["worst_status"] == 0 for st in stats)
    ys = [x.clone() for x in init]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for y, x in zip(ys, init):
            y.copy_(x)
        b.step_async(ys, discs[0].t_span)
    for _ in range(2):
        for y in ys:
            y.zero_()
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        st2 = b.step_wait()
        for i in range(len(discs)):
            assert st2[i]["worst_status"] == 0 and st2[i]["accepted"] == stats[i]["accepted"]
            assert torch.equal(ys[i], refs[i])
    b.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_async_step_in_a_cuda_graph(coag_mod, precision):
    d = synth.make_disc(8, 16, 40, 1e-5, 1.0, 5.0, 100.0, 300.0, alpha=1e-3, v_frag=100.0, seed=35)
    s = torch.cuda.Stream()
    g = coag_mod.Coag(d, precision, stream=s)
    rho0 = g.state(d.rho0)
    ref = rho0.clone()
    with torch.cuda.stream(s):
        st = g.step(ref, d.t_span)
    assert st["status"] == 0
    y = rho0.clone()
    dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        g.step_async(y, d.t_span, dt)
    for _ in range(2):
        with torch.cuda.stream(s):
            y.copy_(rho0)
            dt.zero_()
        graph.replay()
        st2 = g.step_wait()
        assert st2["status"] == 0 and st2["accepted"] == st["accepted"]
        assert torch.equal(y, ref)


def test_full_size_32_disc_batch_sampled(coag_mod, oracle_mod):
    """The 32 uneven discs (~3e5 cells, 40-150 bins) in one batched step of
    the mixed path; two sampled cells per disc against the oracle replay."""
    discs = synth.batch_32_discs()
    t_span = 100.0 * synth.CONST["yr"]
    b = coag_mod.Batch(discs, "mixed")
    recs = [b.disc(i).set_records(4000) for i in range(len(b))]
    ys = [b.disc(i).state(d.rho0) for i, d in enumerate(discs)]
    stats = b.step(ys, t_span)
    for i, d in enumerate(discs):
        assert stats[i]["worst_status"] == 0 and stats[i]["mass_err_max"] < 1e-9
        n = recs[i]["n"].cpu().numpy()
        cells = np.array([0, d.n_cells - 1 - (7 * i) % d.n_cells])
        want = oracle_mod.Oracle(d.subset(cells)).replay(d.rho0[cells], recs[i]["dt"].cpu().numpy()[cells],
                                                         n[cells])
        check_rel(ys[i].cpu().numpy()[cells], want, d.rho0[cells].sum(1), 1e-5)
    b.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_step_host_equals_device_step(coag_mod, precision):
    """cudisc_coag_step_host (host buffers in and out, kernel rebuilt)
    integrates exactly as cudisc_coag_step on a device copy of the state,
    from pinned and from pageable memory, in place or not."""
    d = synth.make_disc(4, 64, 50, 1e-5, 1.0, 5.0, 40.0, 20.0, seed=31)
    g = coag_mod.Coag(d, precision)
    y = g.state(d.rho0)
    ref = g.step(y, d.t_span)
    want = y.cpu().numpy()
    pinned = torch.from_numpy(np.ascontiguousarray(d.rho0)).pin_memory()
    out = torch.empty_like(pinned).pin_memory()
    st = g.step_host(pinned, out, d.t_span)
    assert st["status"] == 0 and st["accepted"] == ref["accepted"]
    assert np.array_equal(out.numpy(), want)
    assert np.array_equal(pinned.numpy(), d.rho0)            # the input is left as it was
    pageable = np.ascontiguousarray(d.rho0).copy()
    st = g.step_host(pageable, pageable, d.t_span, rebuild=False)
    assert st["accepted"] == ref["accepted"] and np.array_equal(pageable, want)
    # the copy-in on the context's second stream, beside the rebuild: from
    # pageable memory in place, then twice in a row from pinned memory
    pageable = np.ascontiguousarray(d.rho0).copy()
    st = g.step_host(pageable, pageable, d.t_span, rebuild=True)
    assert st["accepted"] == ref["accepted"] and np.array_equal(pageable, want)
    for _ in range(2):
        out.zero_()
        st = g.step_host(pinned, out, d.t_span)
        assert st["accepted"] == ref["accepted"] and np.array_equal(out.numpy(), want)
    g.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cost_ordered_slots_change_no_result(coag_mod, precision):
    """With cost_order = 0 the second step hands cells to slots in order of
    the first step's per-cell cost (costliest first); every cell's result,
    step count and step size equal those of index order (cost_order = 1),
    bitwise."""
    d = synth.make_disc(16, 64, 40, 1e-5, 1.0, 5.0, 100.0, 100.0, seed=5, rho_pert=0.1)
    a = coag_mod.Coag(d, precision, cost_order=0)
    b = coag_mod.Coag(d, precision, cost_order=1)
    outs = []
    for g in (a, a, b):
        y = g.state(d.rho0)
        dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
        rec = g.set_records(4000)
        st = g.step(y, d.t_span, dt)
        assert st["status"] == 0
        outs.append((y.clone(), dt.clone(), rec["n"].clone(), st["accepted"], st["rejected"]))
        g.set_records(0)
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1]) and torch.equal(o[2], outs[0][2])
        assert o[3:] == outs[0][3:]
    a.close()
    b.close()
