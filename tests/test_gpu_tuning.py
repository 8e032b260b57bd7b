"""Launch tuning and CUDA graphs of the NTU library on the GPU: every
schedule choice gives the same bond updates bit for bit, the unit-cell step
replayed from its CUDA graph equals the directly launched one, invalid
tunings are refused, and the autotuner picks a valid choice."""
import numpy as np
import pytest

from paper_2107_06635_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_every_tuning_gives_identical_updates():
    """D = 8, split-BF16, 6 items (the context allocates 4-way ALS splits):
    t12 pairing on/off x 2 or 3 ALS CTAs per SM x ALS split 1, 2, 4 give,
    within each build of the reduced metric (lanes, tensor cores), the same
    A', B' and info bit for bit; the two builds agree to 1e-10, and the
    automatic choice reproduces one of them exactly."""
    from paper_2107_06635_gb300 import autotune, ntu
    D, n = 8, 6
    Ta, Tb, G = I.batch_items(21, n, 2, D, I.zz_gate(0.01))
    ctx = ntu.Context(D, 2, 1, 2, 10, ntu.NTU_MIXED_BF16X3, 4, 8, n)
    ref = ctx.batch_update_host(Ta, Tb, G)
    auto, smax = ctx.get_tuning()
    assert auto == autotune.AUTOMATIC and smax == 4
    assert autotune.builds_of(ctx.set_tuning) == (1, 2)
    cands = autotune.candidates(D, ntu.NTU_MIXED_BF16X3, smax, (1, 2))
    assert len(cands) == 12 + 12
    per_build = {}
    for t in cands:
        ctx.set_tuning(**t)
        out = ctx.batch_update_host(Ta, Tb, G)
        first = per_build.setdefault(t["als_build"], out)
        for a, b in zip(out, first):
            assert np.array_equal(a, b), t
    for a, b in zip(per_build[2][:2], per_build[1][:2]):
        assert np.linalg.norm(a - b) < 1e-10 * np.linalg.norm(b)
    assert any(all(np.array_equal(a, b) for a, b in zip(ref, per_build[k])) for k in (1, 2))
    ctx.close()


def test_invalid_tunings_are_refused():
    from paper_2107_06635_gb300 import ntu
    ctx = ntu.Context(4, 2, 1, 2, 10, ntu.NTU_MIXED_BF16X3, 4, 8, 400)
    _, smax = ctx.get_tuning()
    assert smax == 1                      # 400 items: no ALS split allocated
    for bad in ({"t12_pair": 1}, {"als_ctas_per_sm": 4}, {"als_split": 3}, {"als_split": 2},
                {"als_build": 3}, {"als_build": 2}):     # K = D r = 8: no tensor-core build
        with pytest.raises(ntu.NTUError) as e:
            ctx.set_tuning(**bad)
        assert e.value.status == 1, bad
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_step_graph_replay_equals_direct_launches(precision):
    """Three NTU steps and three SU steps of the TFIM quench at D = 4: the
    graph-replayed cell step and the directly launched one give identical
    states, deltas and bond tensors."""
    from paper_2107_06635_gb300 import ntu
    gates2, gate1 = I.tfim_real_time_gates(2.5, 0.01)
    A0, B0 = I.quench_start(4)
    res = []
    for graphs in (True, False):
        ctx = ntu.Context(4, 2, 1, 2, 10, precision, 4, 15 if precision == 0 else 8, 1)
        ctx.set_graphs(graphs)
        ctx.set_state(A0, B0)
        d = [ctx.step(gates2, gate1) for _ in range(3)] + [ctx.step(gates2, None)]
        n_launch = ctx.last_launch_count()
        s = [ctx.su_step(gates2, gate1) for _ in range(3)]
        res.append((ctx.get_state(), np.array(d), np.array(s), ctx.su_get_lambdas(), n_launch))
        ctx.close()
    (sa, da, ta, la, na), (sb, db, tb, lb, nb) = res
    assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
    assert np.array_equal(da, db) and np.array_equal(ta, tb) and np.array_equal(la, lb)
    assert na == nb and na > 40


def test_autotuner_picks_a_valid_choice():
    """The autotuner on a 96-item D = 8 batch: it times every candidate,
    applies one that is no slower than the automatic choice, and the tuned
    context still gives the automatic choice's results (to the agreement of
    the two reduced-metric builds)."""
    from paper_2107_06635_gb300 import autotune, ntu
    D, n = 8, 96
    Ta_h, Tb_h, G_h = I.batch_items(22, n, 2, D, I.zz_gate(0.01))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        Ta, Tb, G = (torch.from_numpy(x).cuda() for x in (Ta_h, Tb_h, G_h))
        Ta_o, Tb_o = torch.empty_like(Ta), torch.empty_like(Tb)
        info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
        ctx = ntu.Context(D, 2, 1, 2, 10, ntu.NTU_MIXED_BF16X3, 4, 8, n, stream=stream.cuda_stream)
        ctx.batch_update_dev(n, Ta, Tb, G, Ta_o, Tb_o, info)
        ctx.sync()
        ref = Ta_o.cpu().numpy().copy()
        rec = autotune.tune_batch(ctx, n, Ta, Tb, G, Ta_o, Tb_o, info, stream, reps=2)
        assert rec["chosen_ms"] <= rec["automatic_ms"]
        assert len(rec["table"]) == len(autotune.candidates(D, ntu.NTU_MIXED_BF16X3,
                                                            ctx.get_tuning()[1], (1, 2)))
        ctx.batch_update_dev(n, Ta, Tb, G, Ta_o, Tb_o, info)
        ctx.sync()
    # the choice may switch the reduced-metric build (lanes / tensor cores),
    # which agree to ~1e-13, not bit for bit
    out = Ta_o.cpu().numpy()
    assert np.linalg.norm(out - ref) <= 1e-10 * np.linalg.norm(ref)
    ctx.close()
