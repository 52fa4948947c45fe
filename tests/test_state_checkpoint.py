"""Checkpointing of the optimiser state (SqngdState.save / load): a host-side
round trip that preserves every buffer bit for bit, its dtype and the step
counters, for the filter-optimising and the matched (SQNAF) states."""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import api, workloads as wl


def _state(matched: bool, seed: int = 3):
    M, N = 3, 17
    u = torch.from_numpy(wl.logits(seed, M, N).astype(np.float32))
    h = None if matched else torch.from_numpy(wl.complex_normal(seed, M, N).astype(np.complex64))
    st = api.SqngdState.create(u, h)
    st.m_u.copy_(torch.from_numpy(wl.normal(seed, M * N, 40).reshape(M, N).astype(np.float32)))
    st.v_u.copy_(st.m_u * st.m_u)
    if not matched:
        st.m_h.copy_(torch.from_numpy(wl.complex_normal(seed + 1, M, N).astype(np.complex64)))
        st.v_h.copy_(torch.from_numpy(wl.complex_normal(seed + 2, M, N).astype(np.complex64)))
    st.best_q.copy_(torch.from_numpy(wl.phase_indices(seed, M, N, 400)))
    st.best.copy_(torch.tensor([0.03125, 0.5, 17.0, 0.49], dtype=torch.float64))
    st.t_h, st.t_x, st.outer = 170, 160, 17
    st.stop = [0.0412, 9]
    return st


@pytest.mark.parametrize("matched", [False, True])
def test_save_load_round_trip_is_bit_exact(tmp_path, matched):
    st = _state(matched)
    path = str(tmp_path / "state.npz")
    st.save(path)
    got = api.SqngdState.load(path, device="cpu")
    assert (got.t_h, got.t_x, got.outer) == (st.t_h, st.t_x, st.outer)
    assert got.stop == st.stop
    for k in api.SqngdState._BUFFERS:
        a, b = getattr(st, k), getattr(got, k)
        if a is None:
            assert b is None, k
            continue
        assert a.dtype == b.dtype and a.shape == b.shape, k
        assert torch.equal(a.view(torch.uint8) if a.is_complex() else a, b.view(torch.uint8) if b.is_complex() else b), k
    assert matched == (got.h is None and got.m_h is None and got.v_h is None)
