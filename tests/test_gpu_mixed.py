"""Mixed-precision path (BF16x3 tensor-core pp ladder, FP32 contractions, FP64
denominators/energy) against the FP64 oracle, through the C ABI.

Error bound of one BF16x3 product: with x = hi + lo + d, |hi - x| <= 2^-9 |x|,
|lo| <= 2^-9 |x| and |d| <= 2^-18 |x|, the dropped and rounding terms sum to at most
3 * 2^-18 |V||t| (about 1.2e-5); FP32 accumulation over K <= 1200 terms adds at most
K * 2^-24 relative in the worst case.  The tests use 5e-5 * sum_cd |V||t| per element.
"""
import numpy as np
import pytest

from conftest import minnesota_params
from inputs import random_amplitudes
import spinflip
from oracle import channel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_06765_gb300 import build
    build.build()
    import paper_1611_06765_gb300 as P
    return P


def _blocks(o, t):
    """Per-channel (offset, nhh, npp) of the library layout (hh rows, pp contiguous)."""
    tab = o.channel_tables()
    off = 0
    for c, (nh, np_) in enumerate(zip(tab["nhh"], tab["npp"])):
        yield c, off, int(nh), int(np_)
        off += int(nh) * int(np_)


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 4), (14, 0.08, 20), (66, 0.16, 36)])
def test_pp_ladder_operator(pkg, N, rho, n2):
    g = pkg.Context(N, rho, n2, params=minnesota_params())
    o = channel.OracleSystem(N, rho, n2, minnesota_params())
    n = len(g.amplitude_labels())
    t = random_amplitudes(n, seed=7)
    r64 = g.apply_pp_ladder(t, precision=pkg.PNM_PREC_FP64)
    rf2 = g.apply_pp_ladder(t, precision=pkg.PNM_PREC_F32PAIR)
    r16 = g.apply_pp_ladder(t, precision=pkg.PNM_PREC_BF16X3)
    ref = np.zeros(n)
    bound = np.zeros(n)
    for c, off, nh, npp in _blocks(o, t):
        V = o.vpp_block(c)
        tb = t[off:off + nh * npp].reshape(nh, npp)
        ref[off:off + nh * npp] = (tb @ V).ravel()
        bound[off:off + nh * npp] = (np.abs(tb) @ np.abs(V)).ravel()
    scale = np.max(np.abs(ref))
    assert scale > 0
    assert np.max(np.abs(r64 - ref)) <= 1e-12 * scale
    # FP32 pairs: 48 significant bits, exact products, two-sum accumulation
    print("FP32-pair pp ladder: max |error| / max |ref| = %.3g" % (np.max(np.abs(rf2 - ref)) / scale))
    assert np.max(np.abs(rf2 - ref)) <= 1e-12 * scale
    assert np.max(np.abs(rf2 - r64)) <= 1e-12 * scale
    assert np.all(np.abs(r16 - ref) <= 5e-5 * bound + 1e-30)
    g.close()


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 4), (14, 0.08, 20), (66, 0.16, 36)])
def test_mixed_solve_within_target(pkg, N, rho, n2):
    """E_corr/N of the mixed path after two FP64 refinement sweeps within 1e-6 MeV of the
    FP64 oracle."""
    g = pkg.Context(N, rho, n2, params=minnesota_params())
    o = channel.OracleSystem(N, rho, n2, minnesota_params())
    dE_o, _, _, _ = o.ccd(alpha=0.5, tol=1e-10 * N, maxit=300)
    dE, it, _, rc = g.solve(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-7,
                            max_iter=300, refine_sweeps=2, allow=(pkg.PNM_ENOTCONV,))
    assert abs(dE[0] - dE_o) / N < 1e-6
    g.close()


def test_mixed_then_fp64_agree_on_fixed_point(pkg):
    """Without refinement the mixed fixed point is already within the target; FP64 sweeps
    from it move the energy by less than 1e-6 MeV per particle."""
    N = 14
    g = pkg.Context(N, 0.08, 20, params=minnesota_params())
    dEm, _, _, _ = g.solve(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-8,
                           max_iter=300)
    dE64, _, _, _ = g.solve(precision=pkg.PNM_PREC_FP64, alpha=0.5, tol=1e-30, tol_per_N=1e-8,
                            max_iter=300)
    assert abs(dEm[0] - dE64[0]) / N < 1e-6
    g.close()


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 4), (14, 0.08, 20), (66, 0.16, 36)])
def test_ph_term_operator(pkg, N, rho, n2):
    """The ph term (cross-channel T, chi_kb^cj, Q and P(ij)P(ab)) against the oracle's, on
    seeded amplitudes: FP64 kernels to 1e-12 of the largest element; the mixed kernels (FP32
    operands and accumulation) within 2e-5 of the oracle's absolute-value bound per element
    (two chained FP32 products over at most 66 terms each: at most 2 * 66 * 2^-24 of it)."""
    g = pkg.Context(N, rho, n2, params=minnesota_params())
    o = channel.OracleSystem(N, rho, n2, minnesota_params())
    lab = g.amplitude_labels()
    perm = spinflip.flip_permutation(lab, o.states())
    t = random_amplitudes(len(lab), seed=9)
    ts = spinflip.symmetrise(t, perm)  # the library forms the term of the symmetric part
    ref = o.ph_apply(ts)
    bound = o.ph_apply(ts, absval=True)
    r64 = g.apply_ph_term(t, precision=pkg.PNM_PREC_FP64)
    rf2 = g.apply_ph_term(t, precision=pkg.PNM_PREC_F32PAIR)
    r16 = g.apply_ph_term(t, precision=pkg.PNM_PREC_BF16X3)
    scale = np.max(np.abs(ref))
    assert scale > 0
    assert np.max(np.abs(r64 - ref)) <= 1e-12 * scale
    print("FP32-pair ph term: max |error| / max |ref| = %.3g" % (np.max(np.abs(rf2 - ref)) / scale))
    assert np.max(np.abs(rf2 - ref)) <= 1e-12 * scale
    assert np.max(np.abs(rf2 - r64)) <= 1e-12 * scale
    ratio = np.abs(r16 - ref) / (bound + 1e-300)
    print("mixed ph: max error / element bound = %.3g" % np.max(ratio))
    assert np.all(np.abs(r16 - ref) <= 2e-5 * bound + 1e-30)
    assert np.array_equal(g.apply_ph_term(spinflip.flip(t, perm), precision=pkg.PNM_PREC_FP64), r64)
    g.close()


def test_keep_start_is_symmetrised(pkg):
    """A kept start that is not flip-symmetric converges to the solution from the MBPT2 start
    (the kept amplitudes are symmetrised first), in FP64 and in the mixed path."""
    N, rho, n2 = 14, 0.08, 20
    g = pkg.Context(N, rho, n2, params=minnesota_params())
    o = channel.OracleSystem(N, rho, n2, minnesota_params())
    dE_o, _, _, _ = o.ccd(alpha=0.5, tol=1e-13, maxit=600)
    perm = spinflip.flip_permutation(g.amplitude_labels(), o.states())
    g.solve(alpha=0.5, tol=1e-12, max_iter=600)
    t = g.get_amplitudes()
    assert np.max(np.abs(t - spinflip.flip(t, perm))) <= 1e-12 * np.max(np.abs(t))
    noisy = t + random_amplitudes(len(t), seed=5, scale=2e-3)
    g.set_amplitudes(noisy)
    dE, _, _, _ = g.solve(alpha=0.5, tol=1e-13, max_iter=600, init=pkg.PNM_INIT_KEEP)
    assert abs(dE[0] - dE_o) < 1e-10 * abs(dE_o), (dE[0], dE_o)
    t2 = g.get_amplitudes()
    assert np.max(np.abs(t2 - spinflip.flip(t2, perm))) <= 1e-12 * np.max(np.abs(t2))
    g.set_amplitudes(noisy)
    dE, _, _, _ = g.solve(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-8,
                          max_iter=600, init=pkg.PNM_INIT_KEEP, refine_sweeps=2)
    assert abs(dE[0] - dE_o) / N < 1e-6, (dE[0], dE_o)
    g.close()


@pytest.mark.parametrize("N,rho,n2", [(14, 0.08, 20), (66, [0.05, 0.11, 0.17], 36)])
def test_pair_refinement_matches_fp64_refinement(pkg, N, rho, n2):
    """The refinement sweeps with FP32-pair contractions (PNM_PREC_F32PAIR) end where the
    sweeps with FP64-pipe contractions end: the same number of updates and energies within
    1e-11 relative (the contractions agree to about 1e-13 of their largest element, the update,
    denominators, residual and energy are FP64 in both), and within 1e-6 MeV per neutron of the
    oracle's fixed point."""
    P = minnesota_params()
    g = pkg.Context(N, rho, n2, params=P)
    kw = dict(precision=pkg.PNM_PREC_BF16X3, alpha=0.5, tol=1e-30, tol_per_N=1e-6, max_iter=300, refine_sweeps=2)
    dE64, it64, _, _ = g.solve(refine_kernels=pkg.PNM_PREC_FP64, **kw)
    dEf2, itf2, _, _ = g.solve(refine_kernels=pkg.PNM_PREC_F32PAIR, **kw)
    assert np.array_equal(it64, itf2), (it64, itf2)
    assert np.all(np.abs(dEf2 - dE64) <= 1e-11 * np.abs(dE64)), (dEf2, dE64)
    rhos = np.atleast_1d(rho)
    for k, r in enumerate(rhos):
        o = channel.OracleSystem(N, r, n2, P)
        dE_o, _, _, _ = o.ccd(alpha=0.5, tol=1e-10 * N, maxit=400)
        assert abs(dEf2[k] - dE_o) / N < 1e-6
    g.close()
