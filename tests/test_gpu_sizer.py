"""The learned sizer on the GPU: exact labels, features and gradients against
the CPU references, and what the trained network gains over sizing without
it."""
import numpy as np
import pytest

import oracle
from oracle import sizer_ref as R
from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg

from .helpers import assert_paths_equal, wrap_digraph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tpg.load_library(build=True)


def load_batch(cfgs):
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    return tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext), int(ns.sum())


def oracle_root_counts(cfgs):
    rows = []
    for c in cfgs:
        r = oracle.run_cfg(c, test_paths=False, want_paths=False)
        rows.append(np.stack([r.root_paths, r.root_pps, r.root_pp_ints], axis=1))
    return np.concatenate(rows)


@pytest.mark.parametrize("which", ["structured-24", "structured-120", "wrapped", "batch-64"])
def test_root_counts_exact(which):
    if which == "structured-24":
        cfgs = [G.config1_cfg()]
    elif which == "structured-120":
        cfgs = [G.config3_cfg()]
    elif which == "wrapped":
        cfgs = [wrap_digraph(G.random_digraph(8, 0.3, 11, self_loops=True))]
    else:
        cfgs = [G.random_cfg(G.BATCH_SEED0 + i) for i in range(64)]
    h, N = load_batch(cfgs)
    with h:
        got = tpg.tpg_root_counts(h, N)
    np.testing.assert_array_equal(got, oracle_root_counts(cfgs))


def test_features_match_reference():
    cfgs = [G.config1_cfg(), G.config3_cfg()] + [G.random_cfg(G.TRAIN_SEED0 + i) for i in range(30)]
    h, N = load_batch(cfgs)
    with h:
        x = tpg.tpg_sizer_features(h, N)
    ref, _ = R.batch_inputs(cfgs)
    np.testing.assert_allclose(x, ref, rtol=1e-6, atol=1e-6)


def test_gradient_matches_reference():
    cfgs = [G.random_cfg(G.TRAIN_SEED0 + i) for i in range(40)]
    X, A = R.batch_inputs(cfgs)
    h, N = load_batch(cfgs)
    with h, tpg.tpg_sizer_create(seed=5) as z:
        tpg.tpg_sizer_add_batch(z, h)
        T = tpg.tpg_sizer_batch_targets(z, 0, N)
        exact = oracle_root_counts(cfgs)
        np.testing.assert_allclose(T, np.log1p(exact.astype(np.float64)), rtol=1e-6)
        rng = np.random.default_rng(1)
        for trial in range(3):
            p = rng.normal(0.0, 0.15, R.NPARAM).astype(np.float32)
            tpg.tpg_sizer_set_params(z, p)
            loss, g = tpg.tpg_sizer_loss_grad(z, 0)
            rl, rg = R.loss_grad(p.astype(np.float64), X, A, T.astype(np.float64), bf=True)
            assert abs(loss - rl) / rl < 5e-3, (loss, rl)
            rel = np.linalg.norm(g - rg) / np.linalg.norm(rg)
            cos = float(np.dot(g, rg) / (np.linalg.norm(g) * np.linalg.norm(rg)))
            assert rel < 2e-2 and cos > 0.999, (rel, cos)
            # every parameter block carries gradient
            for lo, hi in [(R.OFF_W0, R.OFF_B0), (R.OFF_WL, R.OFF_WL + R.LAYER), (R.OFF_WO, R.NPARAM)]:
                assert np.linalg.norm(g[lo:hi]) > 0


def per_graph_totals(pred, cfgs):
    out, base = [], 0
    vol = np.expm1(np.maximum(pred.astype(np.float64), 0.0))
    for c in cfgs:
        out.append(vol[base:base + c.n].sum(0))
        base += c.n
    return np.array(out)


def test_trained_sizer_beats_constant_sizing_and_presizes_exactly():
    train = [[G.random_cfg(G.TRAIN_SEED0 + 1000 + b * 256 + i) for i in range(256)] for b in range(6)]
    held = [G.random_cfg(G.HELDOUT_SEED0 + i) for i in range(512)]
    with tpg.tpg_sizer_create(seed=11) as z:
        tot_nodes, tot_n = 0, 0
        for cfgs in train:
            h, N = load_batch(cfgs)
            with h:
                vol = tpg.tpg_sizer_add_batch(z, h)
            tot_nodes += int(vol[0])
            tot_n += N
        losses = tpg.tpg_sizer_train(z, 60, 3e-3)
        assert losses[-1] < 0.5 * losses[0]
        h, N = load_batch(held)
        with h:
            pred, tot = tpg.tpg_sizer_predict(z, h, N)
    truth = np.array([[c.sum() for c in (r.root_paths, r.root_pps, r.root_pp_ints)]
                      for r in (oracle.run_cfg(c, test_paths=False, want_paths=False) for c in held)], np.float64)
    est = per_graph_totals(pred, held)
    const = np.array([[c.n * tot_nodes / tot_n] for c in held])
    err_sizer = np.mean(np.abs(np.log1p(est[:, 0]) - np.log1p(truth[:, 0])))
    err_const = np.mean(np.abs(np.log1p(const[:, 0]) - np.log1p(truth[:, 0])))
    assert err_sizer < 0.5 * err_const, (err_sizer, err_const)


def test_presized_graph_capture_is_exact():
    train = [[G.random_cfg(G.TRAIN_SEED0 + 5000 + b * 128 + i) for i in range(128)] for b in range(4)]
    held = [G.random_cfg(G.HELDOUT_SEED0 + 1000 + i) for i in range(200)]
    with tpg.tpg_sizer_create(seed=3) as z:
        for cfgs in train:
            h, _ = load_batch(cfgs)
            with h:
                tpg.tpg_sizer_add_batch(z, h)
        tpg.tpg_sizer_train(z, 30, 3e-3)
        ns, rp, col, ent, ext = G.concat_batch(held)
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as ref_h:
            pp = tpg.tpg_prime_paths(ref_h)
            ref_pp = pp.host_arrays()
            pp.free()
            tp = tpg.tpg_test_paths(ref_h)
            ref_tp = tp.host_arrays()
            tp.free()
        for margin in (1.0, 1.5, 4.0):
            with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
                caps = tpg.tpg_sizer_presize(z, h, margin)
                assert np.all(caps > 0)
                tpg.tpg_graph_capture(h)
                pp, tp = tpg.tpg_graph_launch(h)
                for a, b in zip(pp.host_arrays(), ref_pp):
                    np.testing.assert_array_equal(a, b)
                for a, b in zip(tp.host_arrays(), ref_tp):
                    np.testing.assert_array_equal(a, b)
                pp.free()
                tp.free()


def test_presize_keeps_capacities_within_free_memory():
    # an absurd margin asks for far more than the device holds: the
    # capacities are cut to half the free memory and the capture stays exact
    import torch

    train = [G.random_cfg(G.TRAIN_SEED0 + 7000 + i) for i in range(128)]
    held = [G.random_cfg(G.HELDOUT_SEED0 + 3000 + i) for i in range(64)]
    ns, rp, col, ent, ext = G.concat_batch(held)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as ref_h:
        with tpg.tpg_prime_paths(ref_h) as pp, tpg.tpg_test_paths(ref_h) as tp:
            ref_pp, ref_tp = pp.host_arrays(), tp.host_arrays()
    with tpg.tpg_sizer_create(seed=4) as z:
        h, _ = load_batch(train)
        with h:
            tpg.tpg_sizer_add_batch(z, h)
        tpg.tpg_sizer_train(z, 5, 3e-3)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
            caps = tpg.tpg_sizer_presize(z, h, 1e12)
            # the arena alone (8-byte nodes) stays within half the free memory
            assert 8 * int(caps[0]) <= free // 2
            tpg.tpg_graph_capture(h)
            pp, tp = tpg.tpg_graph_launch(h)
            for a, b in zip(pp.host_arrays(), ref_pp):
                np.testing.assert_array_equal(a, b)
            for a, b in zip(tp.host_arrays(), ref_tp):
                np.testing.assert_array_equal(a, b)
            pp.free()
            tp.free()
    torch.cuda.synchronize()
    tpg.tpg_release_cached_memory()
    torch.cuda.empty_cache()


def test_checkpoint_round_trip(tmp_path):
    with tpg.tpg_sizer_create(seed=9) as a, tpg.tpg_sizer_create(seed=10) as b:
        pa = tpg.tpg_sizer_get_params(a)
        assert not np.array_equal(pa, tpg.tpg_sizer_get_params(b))
        path = str(tmp_path / "sizer.bin")
        tpg.tpg_sizer_save(a, path)
        tpg.tpg_sizer_load(b, path)
        np.testing.assert_array_equal(pa, tpg.tpg_sizer_get_params(b))


def test_presized_capture_beats_exact_sizing_on_a_new_batch():
    """What the trained network gains on a batch it has not seen: graph mode
    needs every buffer's capacity before capture.  Without the network those
    capacities come from an exact counting run (a full enumeration); with it,
    from the predicted totals.  Both give byte-equal results; the pre-sized
    cold run (predict + capture + replay) must be faster than the exact-sized
    one (count + capture + replay), and must not fall back (the capacities
    are the calibrated predictions times a margin of 4: a network trained on
    2048 graphs underestimates some batches by more than 2x)."""
    import time

    import torch

    train = [[G.random_cfg(G.TRAIN_SEED0 + 7000 + b * 512 + i) for i in range(512)] for b in range(4)]
    held = [G.random_cfg(G.HELDOUT_SEED0 + 2000 + i) for i in range(1024)]
    ns, rp, col, ent, ext = G.concat_batch(held)
    with tpg.tpg_sizer_create(seed=21) as z:
        for cfgs in train:
            h, _ = load_batch(cfgs)
            with h:
                tpg.tpg_sizer_add_batch(z, h)
        tpg.tpg_sizer_train(z, 40, 3e-3)

        def cold(presize):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
                if presize:
                    tpg.tpg_sizer_presize(z, h, 4.0)
                tpg.tpg_graph_capture(h)  # without pre-sizing: an exact run sizes the capture
                a, b = tpg.tpg_graph_launch(h)
                out = a.host_arrays() + b.host_arrays()
                fb = tpg.tpg_get_stats(h)["graph_fallbacks"]
                a.free()
                b.free()
            torch.cuda.synchronize()
            return time.perf_counter() - t0, out, fb

        cold(True)
        cold(False)  # warm-up of both paths (allocator, module loading)
        t_sized, out_sized, fb = min((cold(True) for _ in range(3)), key=lambda r: r[0])
        t_exact, out_exact, _ = min((cold(False) for _ in range(3)), key=lambda r: r[0])
    assert fb == 0
    for x, y in zip(out_sized, out_exact):
        np.testing.assert_array_equal(x, y)
    assert t_sized < t_exact, (t_sized, t_exact)
