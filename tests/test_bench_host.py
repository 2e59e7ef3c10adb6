"""Host logic of the benchmark's roofline figures (no GPU): the fraction of the batch a launch
processes when converged systems are skipped, and the rule that a measured DRAM traffic figure
is reported only for the workload and kernel source it was captured on."""
import hashlib
import os

import numpy as np

import bench


class _Sizes:
    """Stand-in for a context: only the direct-channel sizes (n_hh, n_pp) per system."""

    def __init__(self, per_sys):
        self.nsys = len(per_sys)
        self._s = [np.array(x, np.int32) for x in per_sys]

    def channels(self, sys=0, kind=0):
        assert kind == 0
        return None, self._s[sys], None


CTX = _Sizes([[[2, 10], [4, 5]], [[3, 4]], [[1, 8], [2, 2]]])
N_T = np.array([2 * 10 + 4 * 5, 3 * 4, 1 * 8 + 2 * 2], float)  # amplitudes per system


def test_all_systems_active_gives_one():
    # mixed updates [10, 9, 9] (+2 sweeps): the update still copies a system converged at the
    # ninth update in the tenth, so all of its 10 launches cover the whole batch
    assert bench.work_fraction(CTX, "k_update_mix", [12, 11, 11], 10, True, 2) == 1.0


def test_contractions_skip_converged_systems():
    # contractions skip a system from the update after the one that met the rule
    got = bench.work_fraction(CTX, "k_ph32", [12, 11, 11], 10, True, 2)
    want = (N_T * np.array([10, 9, 9])).sum() / (N_T.sum() * 10)
    assert abs(got - want) < 1e-15 and got < 1.0


def test_fp64_iteration_counts_every_update():
    # FP64 iteration (no sweeps subtracted): updates [20, 19, 18] in 20 launches; the update
    # kernel covers a system one launch longer than its count, capped at the launch count
    got = bench.work_fraction(CTX, "k_update", [20, 19, 18], 20, False, 0)
    want = (N_T * np.array([20, 20, 19])).sum() / (N_T.sum() * 20)
    assert abs(got - want) < 1e-15


def test_refinement_and_dchi_kernels_cover_the_batch():
    # refinement sweeps reopen every system; k_dchi never skips
    for k in ("k_ph_f2", "k_pp_f2", "k_update", "k_dchi32"):
        assert bench.work_fraction(CTX, k, [12, 11, 11], 2, True, 2) == 1.0


def test_traffic_only_for_its_workload_and_source(monkeypatch):
    k = "k_update_mix"
    path = os.path.join(bench.ROOT, "paper_1611_06765_gb300", "csrc", bench.kernel_source(k))
    with open(path, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()[:16]
    monkeypatch.setitem(bench.TRAFFIC, k, (123.0, digest))
    assert bench.measured_traffic(k, bench.DEFAULT_WORKLOAD) == 123.0
    assert bench.measured_traffic(k, "pnm_N66_rho0.16_n2max36_bf16x3") is None
    # a capture of another version of the source is not reported
    monkeypatch.setitem(bench.TRAFFIC, k, (123.0, "0" * 16))
    assert bench.measured_traffic(k, bench.DEFAULT_WORKLOAD) is None
    assert bench.measured_traffic("k_not_captured", bench.DEFAULT_WORKLOAD) is None


def test_kernel_sources_exist():
    for k in bench.TRAFFIC:
        p = os.path.join(bench.ROOT, "paper_1611_06765_gb300", "csrc", bench.kernel_source(k))
        assert os.path.exists(p), p
