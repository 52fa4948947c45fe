"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/sqngd.h and include/warmstart.h declare, its ctypes
structs match the C layout, and host-side validation rejects bad
configurations before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("sqngd.h", "warmstart.h", "resnet.h")]


def _declared():
    names = set()
    for h in HEADERS:
        names |= set(re.findall(r"^AF_API\s+[\w\s\*]+?\b(\w+)\s*\(", open(h).read(), flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_25728_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("af_init", "af_destroy", "af_loss_grad", "af_loss_grad_xh", "af_ambiguity", "quantize",
              "soft_quantize", "af_project", "sqngd_init", "sqngd_step", "af_eval_hard", "af_sync",
              "af_last_error", "af_set_thresholds", "af_path_of", "ws_create", "ws_destroy", "ws_forward",
              "ws_loss_grad", "ws_train_step", "ws_set_params", "ws_get_params", "ws_param_count"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2604_25728_gb300 import _lib
    names = _declared()
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
        assert n in _lib.SIGNATURES, n
    # nothing else leaks out of the library
    assert exported == set(names)


def test_ctypes_structs_match_c_layout(tmp_path):
    from paper_2604_25728_gb300 import _lib
    src = tmp_path / "layout.c"
    fields_c = [f for f, _ in _lib.AfConfig._fields_]
    fields_s = [f for f, _ in _lib.AfState._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sqngd.h"', '#include "warmstart.h"',
             'int main(void){']
    lines.append('printf("ws_config %zu\\n", sizeof(ws_config));')
    for f, _ in _lib.WsConfig._fields_:
        lines.append(f'printf("ws_config.{f} %zu\\n", offsetof(ws_config, {f}));')
    lines.append('printf("af_config %zu\\n", sizeof(af_config));')
    lines.append('printf("af_state %zu\\n", sizeof(af_state));')
    for f in fields_c:
        lines.append(f'printf("af_config.{f} %zu\\n", offsetof(af_config, {f}));')
    for f in fields_s:
        lines.append(f'printf("af_state.{f} %zu\\n", offsetof(af_state, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(got["ws_config"]) == ctypes.sizeof(_lib.WsConfig)
    for f, _ in _lib.WsConfig._fields_:
        assert int(got[f"ws_config.{f}"]) == getattr(_lib.WsConfig, f).offset, f
    assert int(got["af_config"]) == ctypes.sizeof(_lib.AfConfig)
    assert int(got["af_state"]) == ctypes.sizeof(_lib.AfState)
    for f in fields_c:
        assert int(got[f"af_config.{f}"]) == getattr(_lib.AfConfig, f).offset, f
    for f in fields_s:
        assert int(got[f"af_state.{f}"]) == getattr(_lib.AfState, f).offset, f


def _cfg(**kw):
    from paper_2604_25728_gb300 import _lib
    nu = np.array(kw.pop("nu", [-0.5 + j / 32 for j in range(32)]), dtype=np.float64)
    base = dict(M=2, N=32, B=4, L=nu.size, k_lo=-31, k_hi=31, eps=0.1, snrl_db=0.5, r_n=3, c=300.0,
                pnorm=0.0, path=0, n_h=1, n_x=1, lr_h=0.05, lr_x=1e-3, beta1=0.9, beta2=0.999, adam_eps=1e-8)
    base.update(kw)
    cfg = _lib.AfConfig(**base)
    cfg.nu = nu.ctypes.data_as(_lib.P_double)
    return cfg, nu


@pytest.mark.parametrize("bad", [dict(M=0), dict(M=17), dict(N=1), dict(N=5000), dict(B=1), dict(k_lo=-40),
                                 dict(k_lo=3, k_hi=2), dict(eps=1.5), dict(snrl_db=-1.0), dict(r_n=0),
                                 dict(c=0.0), dict(pnorm=0.5), dict(path=9), dict(n_h=0, n_x=0),
                                 dict(L=0), dict(nu=[0.0, float("nan")]),
                                 dict(matched=1, n_h=1, n_x=1), dict(matched=2, n_h=0)])
def test_init_rejects_bad_config_on_host(lib, bad):
    from paper_2604_25728_gb300 import _lib
    cfg, nu = _cfg(**bad)
    h = ctypes.c_void_p()
    st = lib.af_init(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == _lib.AF_ERR_INVALID_ARG
    assert h.value is None
    assert lib.af_last_error(None).decode() != ""


def test_null_arguments_are_rejected(lib):
    from paper_2604_25728_gb300 import _lib
    assert lib.af_init(None, None, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.af_destroy(None) == _lib.AF_ERR_INVALID_ARG
    assert lib.af_sync(None) == _lib.AF_ERR_INVALID_ARG
    assert lib.af_loss_grad(None, None, None, 0, None, None, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.sqngd_step(None, None, 1, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.af_path_of(None) == -1


def test_warmstart_parameter_count_and_host_validation(lib):
    from oracle import warmstart_oracle as wo
    assert lib.ws_param_count() == wo.flatten(wo.init_params(0)).size
    h = ctypes.c_void_p()
    for bad in [(0, 16), (4, 0), (1 << 12, 1 << 12)]:
        assert lib.ws_create(bad[0], bad[1], None, ctypes.byref(h)) == 1      # AF_ERR_INVALID_ARG
        assert not h.value
    assert lib.ws_destroy(None) == 1


def test_generator_host_validation(lib):
    """rn_* checks that need no device: parameter count, bad sizes, NULLs."""
    from paper_2604_25728_gb300 import _lib
    P = 2048
    assert lib.rn_param_count(P) == 2 * 128 * P + 128 + 5 * (2 * 128 * 128 + 2 * 128) + P
    assert lib.rn_param_count(0) == -1
    h = ctypes.c_void_p()
    assert lib.rn_create(0, None, ctypes.byref(h)) == _lib.AF_ERR_INVALID_ARG and h.value is None
    assert lib.rn_create(70000, None, ctypes.byref(h)) == _lib.AF_ERR_INVALID_ARG
    assert lib.rn_create(16, None, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.rn_last_error(None).decode() != ""
    assert lib.rn_destroy(None) == _lib.AF_ERR_INVALID_ARG
    assert lib.rn_forward(None, None, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.sqngd_attach_generator(None, None, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.af_loss_grad_rho(None, None, None, None, None, None, None) == _lib.AF_ERR_INVALID_ARG
    assert lib.af_project_thresholds(None, None) == _lib.AF_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [dict(train_rho=2), dict(train_rho=1, B=64, r_n=200), dict(train_rho=1, lr_rho=-1.0),
                                 dict(train_rho=1, lr_rho=float("nan"))])
def test_threshold_training_config_rejected_on_host(lib, bad):
    from paper_2604_25728_gb300 import _lib
    cfg, nu = _cfg(**bad)
    h = ctypes.c_void_p()
    assert lib.af_init(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.AF_ERR_INVALID_ARG
    assert h.value is None


def test_context_free_error_messages_are_per_thread(lib):
    """af_init and rn_create failures have no handle to hold their message:
    each thread reads the message of its own last failure."""
    import threading
    from paper_2604_25728_gb300 import _lib
    cfg_m, nu_m = _cfg(M=0)
    cfg_n, nu_n = _cfg(N=1)
    go = threading.Barrier(2)
    got = {}

    def worker(name, cfg, P):
        h = ctypes.c_void_p()
        assert lib.af_init(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.AF_ERR_INVALID_ARG
        assert lib.rn_create(P, None, ctypes.byref(h) if P else None) == _lib.AF_ERR_INVALID_ARG
        go.wait()            # both threads have failed before either reads
        got[name] = (lib.af_last_error(None).decode(), lib.rn_last_error(None).decode())

    ts = [threading.Thread(target=worker, args=("m", cfg_m, 0)),          # rn_create: NULL out
          threading.Thread(target=worker, args=("n", cfg_n, 70000))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert "M must be" in got["m"][0] and "N must be" in got["n"][0]
    assert got["m"][1] == "out is NULL" and got["n"][1] == "P must be in 1..65536"
