"""Checkpoint / restart of the network (Section 3.4) on the GPU.

A run that is checkpointed at an interval boundary and restored into a new
model must continue exactly as the uninterrupted run: same spikes after the
checkpoint step, bit-identical voltages and traces, whether or not NetCon
deliveries are pending at the checkpoint (they are re-derived from the
stored spike history).  A restored model continues with its own external
events, so the network can be resumed with new inputs.  The checkpoint is
in input order, so it also restores under another layout.  Restored runs
are also held to the oracle's uninterrupted run of the same inputs: raster
after the checkpoint bit-exact, voltages within 1e-9 mV."""
import numpy as np
import pytest

from scenarios import network
from oracle import simulate, OracleModel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


def driven(**kw):
    return network(n_cells=160, tstop=40.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0, **kw)


def outputs(md, sc, k0):
    md.cn_sync()
    g, k = md.cn_get_spikes()
    sel = k > k0
    tr = np.stack([md.cn_get_trace(r)[k0:] for r in range(len(sc.rec_node))])
    return g[sel], k[sel], tr, md.cn_get_v()


_oracle = {}


def oracle_run(sc, key):
    """The oracle's uninterrupted run of sc (cached per key)."""
    if key not in _oracle:
        _oracle[key] = simulate(sc)
    return _oracle[key]


def assert_matches_oracle(g, k, tr, v, ref, k0):
    rg, rk = ref.spikes()
    sel = rk > k0
    assert np.array_equal(g, rg[sel]) and np.array_equal(k, rk[sel])
    assert np.max(np.abs(tr - ref.traces()[:, k0:])) <= 1e-9
    assert np.max(np.abs(v - ref.v())) <= 1e-9


def pending_at(sc, ref, k0):
    """NetCon deliveries in flight across step k0: a spike at or before k0
    whose delivery step lies after it."""
    rg, rk = ref.spikes()
    ds = np.floor(np.asarray(sc.netcon_delay) / sc.dt + 0.5).astype(np.int64)
    n = 0
    for gid, step in zip(rg.tolist(), rk.tolist()):
        if step <= k0:
            n += int(np.sum((np.asarray(sc.netcon_src) == gid) & (step + ds > k0)))
    return n


def test_restart_continues_bit_exact(cn):
    sc = driven()
    a = cn.from_scenario(sc)
    a.cn_run(20.0)
    ck = a.cn_checkpoint_save()
    a.cn_run(40.0)
    ga, ka, tra, va = outputs(a, sc, 800)
    assert len(ga) > 10
    b = cn.from_scenario(sc)
    b.cn_checkpoint_load(ck)
    assert b.step == 800
    b.cn_run(40.0)
    gb, kb, trb, vb = outputs(b, sc, 800)
    assert np.array_equal(ga, gb) and np.array_equal(ka, kb)
    assert np.array_equal(tra, trb) and np.array_equal(va, vb)
    # the restored raster holds no spike at or before the checkpoint step
    assert np.all(b.cn_get_spikes()[1] > 800)
    # and the restored run is the oracle's uninterrupted one, with NetCon
    # deliveries pending across the checkpoint
    ref = oracle_run(sc, "driven")
    assert pending_at(sc, ref, 800) > 50
    assert_matches_oracle(gb, kb, trb, vb, ref, 800)


def test_restart_with_new_inputs(cn):
    """The saving model only knew the inputs before 20 ms; the restoring model
    has the full input train and continues as a model that had it all along."""
    full = driven()
    early = driven()
    keep = early.ev_t < 20.0
    early.ev_syn, early.ev_t, early.ev_w = early.ev_syn[keep], early.ev_t[keep], early.ev_w[keep]
    ref = cn.from_scenario(full)
    ref.cn_run(40.0)
    g0, k0, tr0, v0 = outputs(ref, full, 800)
    sav = cn.from_scenario(early)
    sav.cn_run(20.0)
    ck = sav.cn_checkpoint_save()
    res = cn.from_scenario(full)
    res.cn_checkpoint_load(ck)
    res.cn_run(40.0)
    g1, k1, tr1, v1 = outputs(res, full, 800)
    assert len(g0) > 10
    assert np.array_equal(g0, g1) and np.array_equal(k0, k1)
    assert np.array_equal(tr0, tr1) and np.array_equal(v0, v1)
    assert_matches_oracle(g1, k1, tr1, v1, oracle_run(full, "driven"), 800)


@pytest.mark.parametrize("save,load", [("interleaved", "constdepth"), ("constdepth", "interleaved")])
def test_restart_in_reference_layouts_against_oracle(cn, save, load):
    """Saved in one of the paper's node orderings and restored in the other
    (the reference layouts, whose arithmetic follows the oracle's operation
    order), resumed with the full input train after saving with only the
    inputs before 20 ms, with NetCon deliveries in flight across the
    checkpoint: the restored run is the oracle's uninterrupted run -- raster
    after the checkpoint bit-exact, every trace and node voltage within
    1e-9 mV."""
    code = {"interleaved": cn.CN_MAP_INTERLEAVED, "constdepth": cn.CN_MAP_CONSTDEPTH}
    full = driven()
    early = driven()
    keep = early.ev_t < 20.0
    early.ev_syn, early.ev_t, early.ev_w = early.ev_syn[keep], early.ev_t[keep], early.ev_w[keep]
    sav = cn.from_scenario(early, mapping=code[save])
    sav.cn_run(20.0)
    ck = sav.cn_checkpoint_save()
    res = cn.from_scenario(full, mapping=code[load])
    res.cn_checkpoint_load(ck)
    res.cn_run(40.0)
    g, k, tr, v = outputs(res, full, 800)
    ref = oracle_run(full, "driven")
    assert pending_at(full, ref, 800) > 50
    assert len(g) > 10
    assert_matches_oracle(g, k, tr, v, ref, 800)


def test_restart_under_another_layout(cn):
    """Saved with one cell per lane, restored with split cells in tall warps:
    the elimination order differs, so voltages agree to rounding."""
    sc = driven()
    a = cn.from_scenario(sc, mapping=cn.CN_MAP_THREAD)
    a.cn_run(16.0)
    ck = a.cn_checkpoint_save()
    a.cn_run(32.0)
    ga, ka, tra, va = outputs(a, sc, 640)
    b = cn.from_scenario(sc, mapping=48 | cn.CN_MAP_TALL)
    b.cn_checkpoint_load(ck)
    b.cn_run(32.0)
    gb, kb, trb, vb = outputs(b, sc, 640)
    assert np.array_equal(ga, gb) and np.array_equal(ka, kb)
    assert np.max(np.abs(tra - trb)) <= 1e-9 and np.max(np.abs(va - vb)) <= 1e-9
    ref = OracleModel(sc)
    ref.run(1280)
    assert_matches_oracle(gb, kb, trb, vb, ref, 640)


def test_checkpoint_errors(cn):
    sc = driven()
    a = cn.from_scenario(sc)
    a.cn_run(10.5)
    with pytest.raises(cn.CNError) as e:
        a.cn_checkpoint_save()
    assert e.value.status == cn.CN_ESTATE
    a.cn_run(11.0)
    ck = a.cn_checkpoint_save()
    other = cn.from_scenario(network(n_cells=160, tstop=40.0, seed=7))
    with pytest.raises(cn.CNError) as e:
        other.cn_checkpoint_load(ck)
    assert e.value.status == cn.CN_EINVAL
    with pytest.raises(cn.CNError):
        cn.from_scenario(sc).cn_checkpoint_load(ck[:-8])


def test_restart_with_channel_types_and_gaps(cn):
    """The heterogeneous channel workload (gates, calcium, the channel
    currents derived from them) and gap junctions between its cells restart
    bit-identically, and the restored run matches the oracle's
    uninterrupted one.  The run is 8 ms: on this strongly spiking channel
    workload the fast layout's FP64 rounding differences, amplified at the
    upstrokes, reach the 1e-9 mV bar after about 12 ms (1.015e-9 mV
    measured there); the reference layouts, which would hold it longer, do
    not take channel types or gap junctions."""
    import dataclasses
    from scenarios import batched
    sc = batched(n_cells=24, tstop=8.0, n_in=8)
    off = np.asarray(sc.cell_offset)
    a = off[:-2] + 1
    b = off[1:-1] + 1
    sc = dataclasses.replace(sc, gap_node=np.concatenate([a, b]).astype(np.int32),
                             gap_peer=np.concatenate([b, a]).astype(np.int32), gap_g=np.full(2 * len(a), 0.001))
    x = cn.from_scenario(sc)
    x.cn_run(4.0)
    ck = x.cn_checkpoint_save()
    x.cn_run(8.0)
    gx, kx, trx, vx = outputs(x, sc, 160)
    y = cn.from_scenario(sc)
    y.cn_checkpoint_load(ck)
    y.cn_run(8.0)
    gy, ky, try_, vy = outputs(y, sc, 160)
    assert np.array_equal(gx, gy) and np.array_equal(kx, ky)
    assert np.array_equal(trx, try_) and np.array_equal(vx, vy)
    ref = simulate(sc)
    assert len(ref.spikes()[0]) >= 5
    assert_matches_oracle(gy, ky, try_, vy, ref, 160)
    for kind, ncol in (("na3h", 2), ("cahva", 3)):
        n = sc.mech(kind).n
        for col in range(ncol):
            assert np.array_equal(x.cn_get_state(kind, col, n), y.cn_get_state(kind, col, n))
