"""Accuracy of the FP32 and compressed-record forms against the FP64 oracle.

The spike trains of the FP32 plain form, the int8 per-pair form and the bfloat16 form
all diverge from the FP64 reference after a while (the circuit is chaotic), so they are
compared through the statistics §4.1 uses: per-population firing rate and the mean
coefficient of variation of the inter-spike intervals, after discarding an initial
transient (the paper discards the first second).

* test_accuracy_short (always run): 2 s of the full circuit, loose bounds, as a
  regression guard.
* test_accuracy_10s (SNN_ACCURACY=1): 10 s, rate within 2 % and ISI CV within 5 % for
  every population, the stated accuracy target; about 8 minutes of FP64 oracle time.
"""

import os

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2405_02019_gb300 as snn  # noqa: E402


def population_stats(t, i, pop_off, t0, t1, dt_ms=0.1):
    """Per population: rate (Hz) over steps [t0, t1) and the mean ISI CV of neurons with
    at least two intervals in the window."""
    sel = (t >= t0) & (t < t1)
    t, i = t[sel], i[sel]
    order = np.lexsort((t, i))
    t, i = t[order], i[order]
    secs = (t1 - t0) * dt_ms * 1e-3
    rates, cvs = [], []
    for b in range(len(pop_off) - 1):
        lo, hi = pop_off[b], pop_off[b + 1]
        m = (i >= lo) & (i < hi)
        rates.append(m.sum() / ((hi - lo) * secs))
        ti, ii = t[m], i[m]
        isi = np.diff(ti).astype(np.float64)
        same = np.diff(ii) == 0
        isi, owner = isi[same], ii[1:][same] - lo
        cnt = np.bincount(owner, minlength=hi - lo)
        s1 = np.bincount(owner, weights=isi, minlength=hi - lo)
        s2 = np.bincount(owner, weights=isi * isi, minlength=hi - lo)
        ok = cnt >= 2
        if not ok.any():
            cvs.append(np.nan)
            continue
        mean = s1[ok] / cnt[ok]
        var = np.maximum(s2[ok] / cnt[ok] - mean * mean, 0.0)
        cvs.append(float(np.mean(np.sqrt(var) / mean)))
    return np.array(rates), np.array(cvs)


def _gpu_raster(model, wl, steps, fmt):
    net = snn.Network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed, record_format=fmt,
                      raster_capacity=1 << 26)
    net.step(steps)
    t, i = net.read_spikes()
    net.close()
    return t, i


def _compare(steps, discard, rate_tol, cv_tol, pops_min_neurons=0):
    model = workload.microcircuit_model()
    wl = workload.WORKLOADS["pd_full"]
    onet = oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, wl.seed)
    ref_t, ref_i = oracle.Sim(model, onet, wl.seed, fp64=True).run(steps, raster_cap=1 << 26)
    r_ref, c_ref = population_stats(ref_t, ref_i, onet.pop_off, discard, steps)
    report = {"fp64": (r_ref, c_ref)}
    sizes = np.diff(onet.pop_off)
    for name, fmt in (("fp32_plain", snn.RECORD_PLAIN9), ("int8_pair", snn.RECORD_PACKED_I8),
                      ("bf16", snn.RECORD_PACKED_BF16)):
        t, i = _gpu_raster(model, wl, steps, fmt)
        r, c = population_stats(t, i, onet.pop_off, discard, steps)
        report[name] = (r, c)
        keep = sizes >= pops_min_neurons
        rel_r = np.abs(r - r_ref) / r_ref
        rel_c = np.abs(c - c_ref) / c_ref
        print(name, "rate rel err", np.round(rel_r, 4), "cv rel err", np.round(rel_c, 4))
        assert np.all(rel_r[keep] <= rate_tol), (name, rel_r)
        assert np.all(rel_c[keep] <= cv_tol), (name, rel_c)
    return report


def test_accuracy_short():
    """2 s (first 0.5 s discarded): every population within 10 % (rate) and 15 % (CV)."""
    _compare(20000, 5000, 0.10, 0.15)


@pytest.mark.skipif(os.environ.get("SNN_ACCURACY") != "1", reason="10 s FP64 reference: set SNN_ACCURACY=1")
def test_accuracy_10s():
    """10 s (first 1 s discarded, as in §4.1): rate within 2 %, ISI CV within 5 %.  Also
    prints the spread between two FP64 instances (network seeds 1 and 2) as the scale
    against which those errors read (the paper compares simulators against the
    variation between NEST runs, §4.1)."""
    report = _compare(100000, 10000, 0.02, 0.05)
    r_ref, c_ref = report["fp64"]
    for name, (r, c) in report.items():
        print(f"{name:12s} rates {np.round(r, 3)} cv {np.round(c, 3)}")
    model = workload.microcircuit_model()
    wl = workload.WORKLOADS["pd_full"]
    onet2 = oracle.build_network(model, wl.scale_n_permille, wl.scale_k_permille, 2)
    t2, i2 = oracle.Sim(model, onet2, 2, fp64=True).run(100000, raster_cap=1 << 26)
    r2, c2 = population_stats(t2, i2, onet2.pop_off, 10000, 100000)
    print("fp64 seed 2 vs seed 1: rate rel diff", np.round(np.abs(r2 - r_ref) / r_ref, 4),
          "cv rel diff", np.round(np.abs(c2 - c_ref) / c_ref, 4))
