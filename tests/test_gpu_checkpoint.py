"""Checkpoint / resume (amplitudes with a header of N, rho, n2max and a channel-table hash) and
divergence detection on a growing energy change."""
import numpy as np
import pytest

from conftest import minnesota_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def test_checkpoint_round_trip_resumes(pkg, tmp_path):
    """Amplitudes saved after a converged solve load bit for bit into a new context of the same
    systems, and a solve from them (init = PNM_INIT_KEEP) stops at once at the same energy."""
    P = minnesota_params()
    kw = dict(alpha=0.5, tol=1e-30, tol_per_N=1e-10, max_iter=300)
    a = pkg.Context(14, [0.06, 0.12], 20, params=P)
    dE_a, it_a, _, _ = a.solve(**kw)
    path = tmp_path / "t.ckpt"
    a.save_checkpoint(path)
    b = pkg.Context(14, [0.06, 0.12], 20, params=P)
    b.load_checkpoint(path)
    for s in range(2):
        assert np.array_equal(a.get_amplitudes(s), b.get_amplitudes(s))
        assert a.checkpoint_header(s) == b.checkpoint_header(s)
    dE_b, it_b, _, _ = b.solve(init=pkg.PNM_INIT_KEEP, **kw)
    assert np.all(it_b <= 2), it_b
    assert np.all(np.abs(dE_b - dE_a) / 14 < 1e-9), (dE_b, dE_a)
    a.close()
    b.close()


def test_checkpoint_rejects_other_systems(pkg, tmp_path):
    """Another n2max (other channel tables), another density, another number of systems and a
    truncated file are refused with PNM_EINVAL, the held amplitudes left as they were."""
    P = minnesota_params()
    a = pkg.Context(14, [0.06, 0.12], 20, params=P)
    a.solve(alpha=0.5, tol=1e-10, max_iter=300)
    path = tmp_path / "t.ckpt"
    a.save_checkpoint(path)
    raw = path.read_bytes()
    short = tmp_path / "short.ckpt"
    short.write_bytes(raw[:-8])
    for other, f in ((pkg.Context(14, [0.06, 0.12], 16, params=P), path),
                     (pkg.Context(14, [0.06, 0.13], 20, params=P), path),
                     (pkg.Context(14, 0.06, 20, params=P), path),
                     (pkg.Context(14, [0.06, 0.12], 20, params=P), short)):
        before = [other.get_amplitudes(s) for s in range(other.nsys)]
        with pytest.raises(pkg.PnmError) as e:
            other.load_checkpoint(f)
        assert e.value.code == -1
        for s in range(other.nsys):
            assert np.array_equal(before[s], other.get_amplitudes(s))
        other.close()
    a.close()


def test_channel_hash_identifies_the_layout(pkg):
    """The hash depends on the channel tables only: equal for two densities of the same (N,
    n2max), different for another n2max."""
    P = minnesota_params()
    g = pkg.Context(14, [0.06, 0.12], 20, params=P)
    h = pkg.Context(14, 0.06, 16, params=P)
    h0, h1, h2 = g.checkpoint_header(0), g.checkpoint_header(1), h.checkpoint_header(0)
    assert h0["channel_hash"] == h1["channel_hash"] and h0["rho"] != h1["rho"]
    assert h0["channel_hash"] != h2["channel_hash"]
    assert h0["N"] == 14 and h0["Z"] == 0 and h0["n2max"] == 20
    assert h0["n_amplitudes"] == len(g.amplitude_labels(0))
    g.close()
    h.close()


def test_growing_energy_change_reports_divergence(pkg):
    """A start far outside the convergence basin (the converged amplitudes times 1000, where
    the quadratic terms dominate): the energy change grows with every update, and the solve
    returns PNM_EDIVERGED by the |dE| doubling rule after 6 updates, every energy still finite,
    instead of running on until the values overflow or the iteration cap."""
    P = minnesota_params()
    g = pkg.Context(14, 0.08, 20, params=P)
    g.solve(alpha=0.5, tol=1e-10, max_iter=300)
    g.set_amplitudes(1000.0 * g.get_amplitudes(0))
    dE, it, _, rc = g.solve(alpha=0.5, tol=1e-10, max_iter=300, init=pkg.PNM_INIT_KEEP,
                            allow=(pkg.PNM_EDIVERGED, pkg.PNM_ENOTCONV))
    hist = g.history(0)
    print("updates", it, "energies", hist[: it[0] + 1])
    assert rc == pkg.PNM_EDIVERGED
    # caught by the doubling rule (6 consecutive updates), before any value overflowed
    assert it[0] == 6, it
    assert np.all(np.isfinite(hist[: it[0] + 1]))
    g.close()
