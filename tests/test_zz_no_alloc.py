"""eig_gram_noalloc: the Gram product for callers that cannot allocate device
memory while they run (it uses a fixed scratch array built into the library
instead of cudaMallocAsync).  Its result must agree with eig_gram's within
the tolerances of the other Gram parity tests, on two calls in a row (the
second call reuses the scratch the first one left behind).  This file is
collected last so that a failure here cannot hide the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_05572_gb300 import _lib as L  # noqa: E402

RTOL = {L.ARITH_F64: 1e-13, L.ARITH_DF64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _blocks(n, a, b, seed, arith, sym):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, a))
    V = U.copy() if sym else rng.standard_normal((n, b))
    Ud = torch.as_tensor(U, device="cuda")
    Vd = torch.as_tensor(V, device="cuda")
    if arith == L.ARITH_DF64:
        Ud, Vd = L.to_df64(Ud), L.to_df64(Vd)
    return U, V, Ud, Vd


@pytest.mark.parametrize("arith,n,a,b,sym", [(L.ARITH_DF64, 100003, 96, 70, False),
                                             (L.ARITH_F64, 250007, 384, 384, True)])
def test_noalloc_matches_eig_gram_twice(arith, n, a, b, sym):
    for call, seed in enumerate((11, 12)):
        U, V, Ud, Vd = _blocks(n, a, b, seed, arith, sym)
        G_ref = torch.empty(a, b, dtype=torch.float64, device="cuda")
        G_new = torch.full((a, b), float("nan"), dtype=torch.float64, device="cuda")
        L.eig_gram(n, a, b, Ud, a, Vd, b, arith, sym, G_ref, b)
        L.eig_gram_noalloc(n, a, b, Ud, a, Vd, b, arith, sym, G_new, b)
        torch.cuda.synchronize()
        ref, new = G_ref.cpu().numpy(), G_new.cpu().numpy()
        scale = np.abs(U).T @ np.abs(V)
        assert np.all(np.isfinite(new)), call
        assert np.all(np.abs(new - ref) <= 2 * RTOL[arith] * scale), call
        assert np.all(np.abs(new - U.T @ V) <= RTOL[arith] * scale), call


def test_noalloc_rejects_results_larger_than_its_scratch():
    a = b = 1449   # a * b > 2^21 float64 elements
    x = torch.zeros(4, a, dtype=torch.float64, device="cuda")
    G = torch.zeros(a, b, dtype=torch.float64, device="cuda")
    with pytest.raises(L.EigError) as e:
        L.eig_gram_noalloc(4, a, b, x, a, x, b, L.ARITH_F64, False, G, b)
    assert e.value.code == L.EIG_EINVAL
