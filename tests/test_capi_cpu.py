"""The C-ABI library loads on a machine without a GPU, exports every symbol the header
declares, and rejects bad arguments before touching the device.  CPU only."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_00750_b300 as tc
    return tc


def _declared_symbols():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]
    names = set()
    for h in hdrs:
        names |= set(re.findall(r"^TC_API\s+[\w\s\*]+?\b(tc_\w+)\s*\(", open(h).read(), flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for want in ["tc_create_stream", "tc_set_consistency", "tc_process_frame", "tc_destroy"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert len(names) >= 14
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(lib.EXPORTED) <= set(names)


def test_default_consistency_is_the_paper_final_setting(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_params.json")))["final"]
    d = lib.default_consistency()
    assert d["k1"] == pytest.approx(g["k1"]) and d["k2"] == pytest.approx(g["k2"])
    assert d["alpha"] == pytest.approx(g["alpha"]) and d["lam"] == pytest.approx(g["lambda"])


def _weights_blob(tmp_path):
    import synth
    spec = synth.NetSpec(chans=(16, 32, 48), radius=3)
    p = tmp_path / "w.tcw"
    synth.write_weights(str(p), spec, synth.he_weights(spec, seed=0))
    return p


def test_create_stream_rejects_bad_arguments(lib, tmp_path):
    with pytest.raises(lib.TcError) as e:
        lib.Stream(64, 64, "fp32", weights_path=str(tmp_path / "missing.tcw"))
    assert e.value.status == lib.TC_ERR_IO
    bad = tmp_path / "bad.tcw"
    bad.write_bytes(b"XXXX" + b"\0" * 64)
    with pytest.raises(lib.TcError) as e:
        lib.Stream(64, 64, "fp32", weights_path=str(bad))
    assert e.value.status == lib.TC_ERR_IO
    good = _weights_blob(tmp_path)
    truncated = tmp_path / "trunc.tcw"
    truncated.write_bytes(good.read_bytes()[:1000])
    with pytest.raises(lib.TcError) as e:
        lib.Stream(64, 64, "fp32", weights_path=str(truncated))
    assert e.value.status == lib.TC_ERR_IO and "truncated" in str(e.value)
    with pytest.raises(lib.TcError) as e:
        lib.Stream(4, 64, "fp32", weights_path=str(good))      # smaller than 2^levels
    assert e.value.status == lib.TC_ERR_INVALID_ARG
    with pytest.raises(lib.TcError) as e:
        lib.Stream(64, 64, 7, weights_path=str(good))           # not a tc_precision
    assert e.value.status == lib.TC_ERR_INVALID_ARG
    with pytest.raises(lib.TcError) as e:
        lib.Stream(64, 64, "fp32")                                # no weights
    assert e.value.status == lib.TC_ERR_INVALID_ARG


def test_null_and_range_checks(lib):
    so = lib._lib
    assert so.tc_create_stream(None, None, None) == lib.TC_ERR_INVALID_ARG
    assert so.tc_set_consistency(None, None) == lib.TC_ERR_INVALID_ARG
    assert so.tc_process_frame(None, None, None, None, None, None) == lib.TC_ERR_INVALID_ARG
    assert so.tc_destroy(None) == lib.TC_ERR_INVALID_ARG
    assert so.tc_op_correlation(0, None, None, 1, 8, 8, 16, 3, None, None) == lib.TC_ERR_INVALID_ARG
    assert so.tc_op_upsample_flow(None, 1, 4, 4, 3, None, None) == lib.TC_ERR_INVALID_ARG
    c = lib._consistency_struct(k1=1.5)
    # tc_op_consistency validates pointers first, then the parameters; fake non-NULL pointers
    # are never dereferenced on the host and the call fails before any launch.
    p = ctypes.c_void_p(16)
    st = so.tc_op_consistency(p, p, p, p, p, p, p, 8, 8, 8, 8, 1, ctypes.byref(c), p, None, None, None)
    assert st == lib.TC_ERR_INVALID_ARG
    assert b"k1" in so.tc_last_error(None)


def test_server_admission_is_decided_before_any_allocation(lib, tmp_path):
    """HBM-budget admission happens on the host: a budget smaller than one stream's charge
    answers TC_ERR_BUSY without touching the device (this runs on a machine without a GPU)."""
    w = _weights_blob(tmp_path)
    srv = lib.Server(str(w), precision="bf16", hbm_budget_bytes=1 << 20, workers=2, max_streams=4)
    small, big = srv.stream_bytes(64, 64), srv.stream_bytes(1920, 1080)
    assert 0 < small < big and big > (1 << 20)
    assert srv.stream_bytes(128, 128) > small
    with pytest.raises(lib.TcError) as e:
        srv.open(1920, 1080)
    assert e.value.status == lib.TC_ERR_BUSY and "budget" in str(e.value)
    assert srv.bytes_in_use == 0
    with pytest.raises(lib.TcError) as e:
        srv.open(4, 4)
    assert e.value.status == lib.TC_ERR_INVALID_ARG
    srv.destroy()
    with pytest.raises(lib.TcError) as e:
        lib.Server(str(w), workers=0)
    assert e.value.status == lib.TC_ERR_INVALID_ARG


def test_trainer_rejects_bad_arguments(lib, tmp_path):
    import synth
    import paper_2301_00750_b300.train as tr
    spec = synth.NetSpec(chans=(16, 32, 48), radius=3)
    good = tmp_path / "net.tcw"
    synth.write_weights(str(good), spec, synth.he_weights(spec, seed=0))
    for kw, want in [(dict(precision=7), lib.TC_ERR_INVALID_ARG), (dict(batch=0), lib.TC_ERR_INVALID_ARG),
                     (dict(height=60), lib.TC_ERR_INVALID_ARG), (dict(lr=-1.0), lib.TC_ERR_INVALID_ARG)]:
        args = dict(batch=2, height=64, width=64, precision="fp32")
        args.update(kw)
        hp = {k: args.pop(k) for k in list(args) if k in ("lr",)}
        with pytest.raises(lib.TcError) as e:
            tr.Trainer(args["batch"], args["height"], args["width"], args["precision"], weights_path=str(good), **hp)
        assert e.value.status == want, kw
    with pytest.raises(lib.TcError) as e:
        tr.Trainer(2, 64, 64, "fp32", weights_path=str(tmp_path / "missing.tcw"))
    assert e.value.status == lib.TC_ERR_IO
    d = tr.default_hparams()
    assert abs(d["lr"] - 1e-4) < 1e-9 and abs(d["beta1"] - 0.9) < 1e-7 and abs(d["beta2"] - 0.99) < 1e-7
    assert abs(d["weight_decay"] - 4e-4) < 1e-9


def test_training_pairs_carry_their_flow():
    """a(x) = b(x + F(x)) wherever no rectangle occludes: resampling b along F (cubic
    B-spline, the generator's own interpolant) reproduces a there."""
    import numpy as np
    import synth
    yy, xx = np.mgrid[0:128, 0:128].astype(float)
    for seed in range(4):
        a, b, f = synth.training_pair(seed, size=128, max_flow=16.0)
        assert a.shape == b.shape == (3, 128, 128) and f.shape == (2, 128, 128)
        assert np.sqrt((f ** 2).sum(0)).max() <= 16.0 + 1e-4
        back = synth.resample(b, yy + f[1], xx + f[0])
        ok = np.abs(back - a).max(0) < 1e-3
        assert ok.mean() > 0.85, (seed, ok.mean())


def test_fp8_scales_from_amax_is_host_arithmetic(lib):
    """The static E4M3 activation scales are computed behind the C ABI (no device needed):
    margin * amax / 448, zero for an all-zero segment; bad records are rejected."""
    import numpy as np
    amax = np.array([448.0, 1.0, 0.0, 3.5, 1e-3], np.float32)
    got = lib.fp8_scales_from_amax(amax)
    assert np.array_equal(got, (amax / np.float32(448)).astype(np.float32))
    assert got[0] == 1.0 and got[2] == 0.0
    got2 = lib.fp8_scales_from_amax(amax, margin=1.25)
    np.testing.assert_allclose(got2, 1.25 * amax / 448, rtol=1e-6)
    for bad_amax, margin in [([1.0, -1.0], 1.0), ([1.0, float("nan")], 1.0), ([1.0], 0.0), ([1.0], float("inf"))]:
        with pytest.raises(lib.TcError) as e:
            lib.fp8_scales_from_amax(np.array(bad_amax, np.float32), margin)
        assert e.value.status == lib.TC_ERR_INVALID_ARG
