"""Host-side arithmetic of the server (no GPU): the work counts it schedules by, checked
against the LTS schedule written out substep by substep (Alg. 2, Fig. blk_loop: level l
steps at substep n iff n is a multiple of 2^(l_max - l)), and the latency summary.
"""
import numpy as np
import pytest

from paper_2011_10570_gb300 import serve


def active_by_schedule(counts, lmin, lmax, n):
    """octants stepping at substep n, from the activity rule"""
    return sum(counts[l] for l in range(lmin, lmax + 1) if n % (1 << (lmax - l)) == 0)


@pytest.mark.parametrize("lmin,lmax", [(3, 5), (4, 9), (2, 2)])
def test_mean_active_octants_is_the_schedule_average(lmin, lmax):
    rng = np.random.default_rng(lmin * 10 + lmax)
    counts = {l: int(rng.integers(1, 5000)) for l in range(lmin, lmax + 1)}
    levels = np.concatenate([np.full(c, l) for l, c in counts.items()])
    nsub = 1 << (lmax - lmin)
    brute = sum(active_by_schedule(counts, lmin, lmax, n) for n in range(nsub)) / nsub
    assert serve.mean_active_octants(levels) == pytest.approx(brute, rel=1e-12)


@pytest.mark.parametrize("lmin,lmax", [(3, 5), (4, 9)])
def test_node_updates_counts_the_active_suffix(lmin, lmax):
    rng = np.random.default_rng(lmax)
    per_level = [0] * 32
    for l in range(lmin, lmax + 1):
        per_level[l] = int(rng.integers(1, 3000))
    st = {"l_min": lmin, "l_max": lmax, "octants_per_level": per_level}
    nsub = 1 << (lmax - lmin)
    counts = {l: per_level[l] for l in range(lmin, lmax + 1)}
    # a whole macro step: V * sum_l n_l 2^(l - l_min)
    macro = 343 * sum(per_level[l] << (l - lmin) for l in range(lmin, lmax + 1))
    assert serve.node_updates(st, 0, nsub) == macro
    # any window of substeps, starting anywhere in the macro step, wrapping around
    for start in (0, 1, nsub // 2 + 1, nsub - 1):
        for n in (1, 3, nsub + 2):
            brute = 343 * sum(active_by_schedule(counts, lmin, lmax, (start + q) % nsub) for q in range(n))
            assert serve.node_updates(st, start, n) == brute


def test_state_bytes_scale_and_precision():
    a = serve.state_bytes(1000, 2, 0)
    assert serve.state_bytes(2000, 2, 0) == 2 * a
    assert serve.state_bytes(1000, 2, 1) < a          # FP32 stage arrays
    assert serve.state_bytes(1000, 1, 0) < a          # one field
    # at least the two FP64 state copies and four FP64 stages of every node
    assert a >= 1000 * 343 * 2 * 8 * (2 + 4)


def test_summary_percentiles_and_throughput():
    res = [serve.Result(rid=i, arrival=0.0, admitted=0.0, finished=float(i + 1), octants=1, substeps=1,
                        node_updates=10.0) for i in range(100)]
    s = serve.summary(res, wall=50.0)
    assert s["requests"] == 100
    assert s["p50_latency_s"] == pytest.approx(50.5)
    assert s["p99_latency_s"] == pytest.approx(99.01)
    assert s["throughput_node_updates_per_s"] == pytest.approx(1000.0 / 50.0)
    assert s["requests_per_s"] == pytest.approx(2.0)
