"""Sampler pieces that need no GPU: the counter-based generator (library vs an independent
oracle implementation and published known-answer vectors), the product's pure-state
construction vs the oracle's (both from Sec. II), and the conditional-state shortcut vs
Eqs. condV/condR."""
import numpy as np
import pytest

from oracle import gbs as G
from oracle import philox as OP
from paper_2010_15595_gb300 import workloads as W


# Known-answer vectors of Philox4x32-10 (counter, key, output) from the generator's
# reference test set.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_oracle_philox_known_answers(ctr, key, want):
    assert tuple(OP.philox4x32_10(ctr, key)) == want


def test_library_philox_matches_oracle():
    from paper_2010_15595_gb300 import sampler as S
    rng = np.random.default_rng(3)
    for _ in range(200):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64)
        assert list(S.philox4x32(ctr, key)) == OP.philox4x32_10(ctr, key)
    for ctr, key, want in KAT:
        assert tuple(int(x) for x in S.philox4x32(ctr, key)) == want


def test_box_muller_moments():
    z = np.concatenate([OP.chain_normals(s, 0, 64) for s in range(200)])
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.05


def _state(m, seed, r=0.5, sigma=0.3):
    rng = W.rng_for(50, seed)
    U = W.haar_unitary(m, rng)
    rv = np.full(m, r)
    al = W.complex_normal(m, sigma, rng)
    return U, rv, al


@pytest.mark.parametrize("m", [1, 3, 5])
def test_product_state_matches_oracle(m):
    """The product builds B, gamma, p(vac) and the Husimi factor with torch (Sec. II); the
    oracle with numpy. Independent code, same equations."""
    from paper_2010_15595_gb300 import sampler as S
    U, rv, al = _state(m, m)
    st = S.pure_state(U, rv, al, device="cpu")
    V = G.pure_state_covariance(U, rv)
    R = G.means_from_alpha(al)
    B, g, pv = G.pure_B_gamma(V, R)
    assert np.abs(st.B - B).max() < 1e-12
    assert np.abs(st.gamma - g).max() < 1e-12
    assert st.p_vac == pytest.approx(pv, rel=1e-12)
    if m > 1:
        VQ = G.heterodyne_cov(V, list(range(1, m)))
        assert np.abs(st.het_chol @ st.het_chol.T - VQ).max() < 1e-12


def test_conditional_state_shortcut_matches_condV_condR():
    """After heterodyne outcome alpha_B on modes B, the pure conditional state of modes A
    has kernel B_AA and fill vector gamma_A + B_AB conj(alpha_B): checked against the
    covariance route of Eqs. condV/condR (Sec. II)."""
    U, rv, al = _state(5, 9, r=0.6)
    V = G.pure_state_covariance(U, rv)
    R = G.means_from_alpha(al)
    B, g, _ = G.pure_B_gamma(V, R)
    for k in (1, 2, 4):
        A_modes, B_modes = list(range(k)), list(range(k, 5))
        aB = np.array([0.3 - 0.2j, -0.1 + 0.5j, 0.2 + 0.1j, -0.4j][: len(B_modes)])
        Vk, Rk = G.conditional_state(V, R, A_modes, B_modes, G.mu_from_alpha(aB))
        Bk, gk, _ = G.pure_B_gamma(Vk, Rk)
        assert np.abs(Bk - B[np.ix_(A_modes, A_modes)]).max() < 1e-12
        shortcut = g[A_modes] + B[np.ix_(A_modes, B_modes)] @ np.conj(aB)
        assert np.abs(gk - shortcut).max() < 1e-12


def _lossy(m, seed, eta):
    from paper_2010_15595_gb300 import sampler as S
    U, rv, al = _state(m, seed, r=0.5, sigma=0.3)
    return S.lossy_state(U, rv, al, eta), (U, rv, al)


@pytest.mark.parametrize("eta", [1.0, 0.6])
def test_williamson_decomposition(eta):
    """Eq. split: V = T + W with T = S^T S pure (S symplectic) and W >= 0."""
    import torch
    from paper_2010_15595_gb300 import sampler as S
    (V, R), _ = _lossy(3, 4, eta)
    Sm, nu = S.williamson(torch.from_numpy(V))
    Sm, nu = Sm.numpy(), nu.numpy()
    m = 3
    Om = np.block([[np.zeros((m, m)), np.eye(m)], [-np.eye(m), np.zeros((m, m))]])
    assert np.abs(Sm @ Om @ Sm.T - Om).max() < 1e-10
    assert np.abs(Sm.T @ np.diag(np.concatenate([nu, nu])) @ Sm - V).max() < 1e-10
    assert (nu >= 1 - 1e-10).all()
    if eta == 1.0:
        assert np.abs(nu - 1).max() < 1e-10
    st = S.mixed_state(V, R, device="cpu")
    W = st.w_factor @ st.w_factor.T
    assert np.linalg.eigvalsh(W).min() > -1e-10


def test_mixed_builder_reduces_to_pure_builder():
    """For a pure state the mixture has W = 0, and the fill map at R-bar gives the pure
    state's fill vector, with the same kernel matrix."""
    from paper_2010_15595_gb300 import sampler as S
    (V, R), (U, rv, al) = _lossy(4, 5, 1.0)
    mx = S.mixed_state(V, R, device="cpu")
    pu = S.pure_state(U, rv, al, device="cpu")
    assert np.abs(mx.w_factor).max() < 1e-6
    assert np.abs(mx.fill_map @ mx.mean - pu.gamma).max() < 1e-10
    assert np.abs(mx.B - pu.B).max() < 1e-10
    assert np.abs(mx.het_chol - pu.het_chol).max() < 1e-8


def test_oracle_threshold_output_is_clicks_of_photon_sample():
    """The oracle's threshold output is min(s_i, 1) of the photon-number sample drawn from
    the same random numbers."""
    import numpy as np
    from oracle import gbs as G
    from paper_2010_15595_gb300 import workloads as W
    rng = W.rng_for(94, 0)
    U = W.haar_unitary(3, rng)
    V = G.pure_state_covariance(U, np.array([0.9, 0.7, 0.5]))
    R = G.means_from_alpha(W.complex_normal(3, 0.3, rng))
    r2 = np.random.default_rng(5)
    for _ in range(10):
        z, u = r2.standard_normal(4), r2.random(3)
        s, _ = G.chain_rule_sample(V, R, 5, z, u)
        t, _ = G.chain_rule_sample(V, R, 5, z, u, threshold=True)
        assert t == [min(x, 1) for x in s]
