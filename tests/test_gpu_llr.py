"""GPU parity of the locally-low-rank prox (pp_prox_llr; the LLR regulariser
of the MRF experiment, Sec. 5.3) against the FP64 oracle's block SVDs:
relative L2 <= 1e-5 per call, for 2-D and 3-D volumes, block edges 4/8/16,
1 to 8 coefficient images, shifted block grids, in place and not, and the
degenerate cases (zero blocks, lambda = 0, lambda above every singular
value)."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pp():
    from paper_2204_10252_gb300.build import build_library
    build_library()
    import paper_2204_10252_gb300 as m
    m.lib()
    return m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def low_rank_images(shape, T, seed):
    """T coefficient images whose blocks have spread singular values: a
    smooth rank-2 part plus noise (an MRF-like subspace image stack)."""
    rng = np.random.default_rng(seed)
    base = [synth.phantom(shape, seed + i).astype(np.complex128) for i in range(2)]
    mix = rng.standard_normal((T, 2)) + 1j * rng.standard_normal((T, 2))
    x = np.einsum("tk,k...->t...", mix, np.stack(base))
    x += 0.05 * np.stack([synth.crandn(shape, seed + 10 + t) for t in range(T)])
    return x.astype(np.complex64)


def lam_between(x, block, shift=None):
    """A lambda inside the range of the blocks' singular values."""
    M, _ = O.llr_blocks(x.astype(np.complex128), block, shift)
    sv = np.concatenate([np.linalg.svd(m, compute_uv=False) for m in M[:64]])
    return float(np.quantile(sv, 0.6))


CASES = [((8, 16, 24), 5, 8, None), ((16, 16, 16), 8, 8, (3, 7, 5)), ((16, 16, 8), 1, 8, None),
         ((32, 48), 5, 8, (5, 0)), ((12, 20), 3, 4, (1, 2)), ((32, 32), 2, 16, None),
         ((8, 12, 16), 4, 4, (2, 3, 1)), ((16, 8, 8), 7, 8, (0, 0, 9))]
IDS = ["3d_8x16x24_T5", "3d_16^3_T8_shift", "3d_16x16x8_T1", "2d_32x48_T5_shift", "2d_12x20_T3_b4",
       "2d_32_T2_b16", "3d_8x12x16_T4_b4", "3d_16x8x8_T7_zshift"]


@pytest.mark.parametrize("case", range(len(CASES)), ids=IDS)
@pytest.mark.parametrize("inplace", [False, True])
def test_llr_prox_matches_oracle(pp, case, inplace):
    import torch
    shape, T, block, shift = CASES[case]
    x = low_rank_images(shape, T, 40 + case)
    lam = lam_between(x, block, shift)
    ref = O.prox_llr(x.astype(np.complex128), lam, block, shift)
    xin = dev(x)
    out = xin if inplace else torch.empty_like(xin)
    pp.pp_prox_llr(shape, T, block, lam, xin, out, shift=shift)
    got = host(out)
    assert rel(got, ref) <= TOL_APPLY
    # thresholding was active and not total
    assert 0 < np.linalg.norm(ref) < np.linalg.norm(x)


def test_llr_prox_degenerate_cases(pp):
    import torch
    shape, T = (16, 16, 8), 5
    x = low_rank_images(shape, T, 3)
    x[:, :8, :8, :8] = 0                 # one all-zero block
    xin = dev(x)
    out = torch.empty_like(xin)
    pp.pp_prox_llr(shape, T, 8, 0.0, xin, out)            # lambda = 0: identity
    got = host(out)
    assert np.all(np.isfinite(got))
    assert rel(got, x.astype(np.complex128)) <= TOL_APPLY
    assert np.all(got[:, :8, :8, :8] == 0)
    pp.pp_prox_llr(shape, T, 8, 1e9, xin, out)            # above every singular value: 0
    assert np.all(host(out) == 0)
    with pytest.raises(pp.PPError) as e:                  # 12 is not a multiple of 8
        pp.pp_prox_llr((12, 16, 8), T, 8, 1.0, dev(np.zeros((T, 12, 16, 8), np.complex64)),
                       torch.empty(T * 12 * 16 * 8, dtype=torch.complex64, device="cuda"))
    assert e.value.status == 2


def test_llr_prox_mrf_sized_volume(pp):
    # an MRF-like stack: 5 coefficient images of 128 x 128 x 128, 8^3 blocks
    # (4096 blocks), against the oracle block by block
    import torch
    shape, T = (128, 128, 128), 5
    x = low_rank_images(shape, T, 77)
    lam = lam_between(x, 8)
    xin = dev(x)
    out = torch.empty_like(xin)
    pp.pp_prox_llr(shape, T, 8, lam, xin, out, shift=(4, 4, 4))
    got = host(out)
    ref = O.prox_llr(x.astype(np.complex128), lam, 8, (4, 4, 4))
    assert rel(got, ref) <= TOL_APPLY
