"""Algorithm 1's stopping test (sqngd_run) and checkpoint/resume on the GPU.

- The run stops exactly where the oracle's reading of the stopping test
  (oracle.stop_rule) stops on the same sequence of hard WPSL values, and its
  results equal those of sqngd_step over the same number of iterations.
- k outer iterations, a checkpoint, a fresh context (and generator) loaded
  from it, and k more iterations equal 2k uninterrupted iterations bit for
  bit: every state buffer, the loss logs, the thresholds and their moments
  (trained thresholds) and the generator's parameters and moments.
"""
import numpy as np
import pytest
import torch

from paper_2604_25728_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_25728_gb300 import api as a
    return a


def _bits(t):
    t = t.detach().contiguous()
    return t.view(torch.uint8) if t.is_complex() else t


def _ctx(api, w, **kw):
    args = dict(eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n, c=w.c, n_h=w.n_h, n_x=w.n_x, lr_h=w.lr_h, lr_x=w.lr_x)
    args.update(kw)
    return api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, **args)


def _fresh(api, ctx, w, seed):
    b = torch.from_numpy(wl.phase_indices(seed, w.M, w.N, w.B)).cuda()
    u, h = ctx.sqngd_init(b)
    return api.SqngdState.create(u, h)


@pytest.mark.parametrize("patience", [3, 12])
def test_sqngd_run_stops_where_the_rule_says(api, orc, patience):
    w = wl.tiny()
    ctx = _ctx(api, w, lr_x=5e-3)
    st = _fresh(api, ctx, w, 4)
    log, stopped = ctx.sqngd_run(st, 400, patience=patience)
    n = log.shape[0]
    assert n == st.outer and stopped in (1, 2)
    exp = orc.stop_rule(log[:, 0, 1], patience, 400)
    assert (n, stopped, st.stop[0], st.stop[1]) == exp
    if stopped == 1:
        assert n - 1 - st.stop[1] == patience          # the patience-th iteration without improvement is the last
        assert np.all(log[st.stop[1] + 1:, 0, 1] >= st.stop[0])
    # the same number of iterations through sqngd_step gives the same bits
    ref = _fresh(api, ctx, w, 4)
    ref_log = ctx.sqngd_step(ref, n)
    assert np.array_equal(ref_log, log)
    for k in ("u", "h", "m_u", "v_u", "m_h", "v_h", "best", "best_q", "best_h"):
        assert torch.equal(_bits(getattr(st, k)), _bits(getattr(ref, k))), k
    ctx.close()


def test_sqngd_run_resumes_the_rule_across_calls(api, orc):
    """Two calls with a t_max between them apply the rule as one call."""
    w = wl.tiny()
    ctx = _ctx(api, w, lr_x=5e-3)
    a = _fresh(api, ctx, w, 6)
    log_a, stop_a = ctx.sqngd_run(a, 300, patience=8)
    b = _fresh(api, ctx, w, 6)
    log_b1, s1 = ctx.sqngd_run(b, 17, patience=8)
    logs = [log_b1]
    if s1 == 2:
        log_b2, s2 = ctx.sqngd_run(b, 300, patience=8)
        logs.append(log_b2)
    else:
        s2 = s1
    assert np.array_equal(np.concatenate(logs), log_a) and s2 == stop_a
    assert b.outer == a.outer and b.stop == a.stop
    ctx.close()


def _run_pair(api, w, tmp_path, k, make_ctx, make_gen=None):
    """2k uninterrupted iterations against k, checkpoint, reload into a fresh
    context (and generator), k more."""
    def setup():
        ctx = make_ctx()
        st = _fresh(api, ctx, w, 9)
        gen = None
        if make_gen is not None:
            gen, y0, u0 = make_gen()
            ctx.attach_generator(gen, y0)
            st.u.copy_(u0)
            ctx._y0 = y0
        return ctx, st, gen

    ctx_a, a, gen_a = setup()
    log_a = ctx_a.sqngd_step(a, 2 * k)

    ctx_b, b, gen_b = setup()
    log_b1 = ctx_b.sqngd_step(b, k)
    path = str(tmp_path / "ck.npz")
    b.save(path, ctx=ctx_b, generator=gen_b)
    ctx_b.close()
    if gen_b is not None:
        gen_b.close()

    ctx_c = make_ctx()
    gen_c, y0 = None, None
    if make_gen is not None:
        gen_c, y0, _ = make_gen()
        ctx_c.attach_generator(gen_c, y0)
        ctx_c._y0 = y0
    c = api.SqngdState.load(path, device="cuda", ctx=ctx_c, generator=gen_c, y0=y0)
    log_c2 = ctx_c.sqngd_step(c, k)

    assert np.array_equal(np.concatenate([log_b1, log_c2]), log_a)
    assert (c.t_h, c.t_x, c.outer) == (a.t_h, a.t_x, a.outer)
    for key in api.SqngdState._BUFFERS:
        assert torch.equal(_bits(getattr(c, key)), _bits(getattr(a, key))), key
    ra, rc = ctx_a.get_rho_state(), ctx_c.get_rho_state()
    for i in range(3):
        assert np.array_equal(ra[i], rc[i])
    assert ra[3] == rc[3]
    if make_gen is not None:
        assert np.array_equal(gen_a.get_params(), gen_c.get_params())
        for x, y in zip(gen_a.get_adam(), gen_c.get_adam()):
            assert np.array_equal(x, y)
        gen_a.close()
        gen_c.close()
    ctx_a.close()
    ctx_c.close()


def test_resume_is_bit_exact_plain(api, tmp_path):
    w = wl.tiny()
    _run_pair(api, w, tmp_path, 15, lambda: _ctx(api, w))


def test_resume_is_bit_exact_trained_thresholds(api, tmp_path):
    w = wl.small(2, 64, 4, 64, r_n=20)
    _run_pair(api, w, tmp_path, 12, lambda: _ctx(api, w, train_rho=True, lr_rho=1e-4))


def test_resume_is_bit_exact_with_generator(api, tmp_path):
    w = wl.tiny()
    P = w.M * w.N
    b = wl.phase_indices(9, w.M, w.N, w.B)
    z0 = ((w.r_n // 2) * w.B + b.astype(np.float64)) / (w.B * w.r_n)

    def make_gen():
        from paper_2604_25728_gb300 import generator
        gen = api.ResNetGenerator(P)
        gen.set_params(generator.init_params(P, z0, 5))
        y0 = torch.from_numpy((b.astype(np.float32) / w.B).ravel()).cuda()
        u0 = gen.forward(y0).reshape(w.M, w.N).contiguous()
        return gen, y0, u0

    _run_pair(api, w, tmp_path, 10, lambda: _ctx(api, w, lr_x=1e-4), make_gen)
