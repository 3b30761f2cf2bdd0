"""The allocation-free entry point peps_cu0_noalloc, checked against the
existing peps_env_cluster.

Callers that cannot allocate device memory (an allocator that already holds
the memory, a latency-critical loop, a framework that forbids allocation)
get the CU_0 separable boundaries from peps_cu0_noalloc, whose scratch is a
static device array.  Two checks, each over two calls in a row (every call
reuses the same scratch):

* the matrices themselves against the FP64 oracle's CU_0 sweep (Section 5.1),
  including a case whose sizes fill the whole scratch array (d=4, D=8, Lx=64);
* with n = 1 every cluster window is a single site closed by exactly these
  boundaries on its four sides, so the site density matrices of
  peps_env_cluster(n=1) must follow from the new call's output.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_6696_gb300 import peps
    return torch, peps


def _orientations(A):
    """Dense lattices whose top-down sweeps are the top, bottom, left and
    right sweeps of A (legs [s, u, l, n, r])."""
    flip = A[::-1].transpose(0, 1, 2, 5, 4, 3, 6)          # rows reversed, u <-> n
    tr = A.transpose(1, 0, 2, 4, 3, 6, 5)                  # rows <-> columns, u <-> l, n <-> r
    trflip = tr[::-1].transpose(0, 1, 2, 5, 4, 3, 6)
    return [np.ascontiguousarray(a) for a in (A, flip, tr, trflip)]


def _sigmas(torch, peps, A, stream):
    out = []
    for Ao in _orientations(A):
        Ly, Lx, d, D = Ao.shape[:4]
        a = torch.from_numpy(Ao).cuda()
        s = torch.zeros((Ly, Lx, D, D), dtype=torch.float64, device="cuda")
        peps.cu0_noalloc(a, s, stream=stream)
        out.append(s.cpu().numpy())
    return out


def _site_rhos(A, sig):
    Ly, Lx, d, D = A.shape[:4]
    sT, sB, sL, sR = sig
    rhos = []
    for y in range(Ly):
        for x in range(Lx):
            du = 1 if y == 0 else D
            dl = 1 if x == 0 else D
            dn = 1 if y == Ly - 1 else D
            dr = 1 if x == Lx - 1 else D
            a = A[y, x, :, :du, :dl, :dn, :dr]
            T = sT[y, x, :du, :du]
            B = sB[Ly - 1 - y, x, :dn, :dn]
            L = sL[x, y, :dl, :dl]
            R = sR[Lx - 1 - x, y, :dr, :dr]
            r = np.einsum("sulnr,tvmoq,uv,lm,no,rq->st", a, a, T, L, B, R)
            rhos.append(r / np.trace(r))
    return np.array(rhos)


def test_noalloc_cu0_matches_cluster_n1_two_calls(env):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(6, 5, 2, 3, seed=77)
    ref = peps.env_cluster(A, n=1, chi=8, mode="var").rho("site")
    ref = ref / np.trace(ref, axis1=1, axis2=2)[:, None, None]
    stream = torch.cuda.current_stream()
    for _ in range(2):
        got = _site_rhos(A, _sigmas(torch, peps, A, stream))
        err = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2))
        assert err < TOL, err


@pytest.mark.parametrize("Ly,Lx,d,D,seed", [(6, 5, 2, 3, 77), (3, 64, 4, 8, 78)])
def test_noalloc_cu0_matches_the_oracle_two_calls(env, Ly, Lx, d, D, seed):
    """sigma[r][x] of every cut against the oracle's top-down CU_0 sweep; the
    second case needs 8 + 3 d D^4 + 4 Lx D^2 + D^2 = 65,608 words, the whole
    static scratch."""
    torch, peps = env
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(Ly, Lx, d, D, seed=seed)
    ref = O.cu0_sweep(O.lattice_from_dense(A))
    a = torch.from_numpy(A).cuda()
    for _ in range(2):
        s = torch.full((Ly, Lx, D, D), 7.0, dtype=torch.float64, device="cuda")
        peps.cu0_noalloc(a, s, stream=torch.cuda.current_stream())
        got = s.cpu().numpy()
        for r in range(Ly):
            for x in range(Lx):
                m = ref[r][x]
                k = m.shape[0]
                assert np.all(got[r, x, k:, :] == 0.0) and np.all(got[r, x, :, k:] == 0.0)
                err = np.max(np.abs(got[r, x, :k, :k] - m))
                assert err < TOL, (r, x, err)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, peps = env
    a = torch.zeros((2, 2, 2, 9, 9, 9, 9), dtype=torch.float64, device="cuda")
    s = torch.zeros((2, 2, 9, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(peps.PepsError) as e:
        peps.cu0_noalloc(a, s)
    assert e.value.code == peps.EINVAL and "static scratch" in str(e.value)
