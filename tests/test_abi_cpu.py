"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/peps.h declares, and fails loudly (no CPU fallback) without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "peps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(peps_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("peps_env_full", "peps_env_cluster", "peps_expect_local", "peps_norm",
              "peps_env_free", "peps_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1311_6696_gb300 import peps
    for n in _declared():
        assert hasattr(peps.lib, n), n
    assert set(_declared()) <= set(peps.EXPORTS) | {n for n in _declared() if hasattr(peps.lib, n)}


def test_no_gpu_means_a_loud_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1311_6696_gb300 import peps, synth
    with pytest.raises(peps.PepsError) as e:
        peps.env_full(synth.workload("4x4_D2"), chi=4)
    assert e.value.code == peps.ECUDA


def test_bond_caps_rule_matches_oracle():
    """The host-side cap rule is reimplemented in C++; check the Python oracle's
    rule on hand-worked cases (so a change to either shows up)."""
    from oracle import peps_oracle as O
    assert O.bond_caps([4, 4, 4, 4], [4, 16, 4], 16) == [4, 16, 4]
    assert O.bond_caps([16] * 10, [256] * 9, 64) == [16, 64, 64, 64, 64, 64, 64, 64, 16]
    assert O.bond_caps([1, 1], [1], 8) == [1]
    assert O.bond_caps([4, 4, 4], [16, 16], 2) == [2, 2]


def test_cu0_noalloc_wrapper_rejects_bad_inputs_before_any_launch():
    """The C side of peps_cu0_noalloc trusts the sizes it is given, so the
    binding checks rank, shapes, dtype, contiguity and device first (each case
    here fails on the host, before the library is called)."""
    torch = pytest.importorskip("torch")
    from paper_1311_6696_gb300 import peps
    f64 = torch.float64
    good_A = torch.zeros((3, 4, 2, 3, 3, 3, 3), dtype=f64)
    good_s = torch.zeros((3, 4, 3, 3), dtype=f64)
    cases = [
        (torch.zeros((3, 4, 2, 3, 3, 3), dtype=f64), good_s, ValueError),          # rank 6
        (torch.zeros((3, 4, 2, 3, 3, 2, 3), dtype=f64), good_s, ValueError),       # ragged legs
        (good_A, torch.zeros((3, 4, 3, 2), dtype=f64), ValueError),               # sigma shape
        (good_A.float(), good_s, TypeError),                                       # float32 A
        (good_A, good_s.float(), TypeError),                                       # float32 sigma
        (good_A.transpose(0, 1).contiguous().transpose(0, 1), good_s, ValueError),  # not contiguous
    ]
    if not torch.cuda.is_available():
        cases.append((good_A, good_s, ValueError))                                 # host tensors
    for A, s, exc in cases:
        with pytest.raises(exc):
            peps.cu0_noalloc(A, s)


def test_iteration_caps_are_validated_on_the_host():
    from paper_1311_6696_gb300 import peps
    for bad in ((-1, 0), (0, -5), (2_000_000, 0)):
        with pytest.raises(peps.PepsError) as e:
            peps.set_iteration_caps(*bad)
        assert e.value.code == peps.EINVAL
    peps.set_iteration_caps(5, 7)
    peps.set_iteration_caps(0, 0)                   # back to the defaults


def test_wait_selftest_without_gpu_is_ecuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1311_6696_gb300 import peps
    with pytest.raises(peps.PepsError) as e:
        peps.wait_selftest(1000)
    assert e.value.code == peps.ECUDA
