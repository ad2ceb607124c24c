"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports
every function include/gsopt.h declares, the Python binding mirrors the C
struct layouts, and the host-only entry points behave (status names, the
N_I rule, argument validation that rejects before touching the device)."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "gsopt.h"


@pytest.fixture(scope="module")
def G():
    from paper_2601_16736_gb300 import build
    build.build()
    from paper_2601_16736_gb300 import gsopt
    return gsopt


def _declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(gs_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_function_is_exported_and_bound(G):
    names = _declared_functions()
    assert len(names) >= 15
    lib = G.lib()
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert hasattr(G, n) or n == "gs_status_string", f"binding lacks {n}"


def test_struct_layouts_match_header(tmp_path, G):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "gsopt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(gs_opt_config), sizeof(gs_camera), sizeof(gs_step_params),
         sizeof(gs_attrs), sizeof(gs_grads));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", offsetof(gs_opt_config, prec), offsetof(gs_opt_config, n_pixels),
         offsetof(gs_step_params, restate_ratio), offsetof(gs_step_params, n_visible),
         offsetof(gs_step_params, noise), offsetof(gs_step_params, aiu_scale), offsetof(gs_step_params, n_active));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = list(map(int, out))
    assert sizes[:5] == [ctypes.sizeof(G.gs_opt_config), ctypes.sizeof(G.gs_camera), ctypes.sizeof(G.gs_step_params),
                         ctypes.sizeof(G.gs_attrs), ctypes.sizeof(G.gs_grads)]
    assert sizes[5:] == [G.gs_opt_config.prec.offset, G.gs_opt_config.n_pixels.offset,
                         G.gs_step_params.restate_ratio.offset, G.gs_step_params.n_visible.offset,
                         G.gs_step_params.noise.offset, G.gs_step_params.aiu_scale.offset,
                         G.gs_step_params.n_active.offset]


def test_status_strings_and_version(G):
    assert G.gs_abi_version() == 2
    assert G.status_name(G.GS_OK) == "GS_OK"
    assert G.status_name(G.GS_ERR_INVALID_ARG) == "GS_ERR_INVALID_ARG"
    assert G.status_name(99) == "GS_ERR_UNKNOWN"


def test_n_i_rule_matches_oracle(G, orc):
    for n in [1, 7, 999, 1000, 640000, 800 * 800, 1920 * 1080, 1234567, 10 ** 9 + 7]:
        assert G.gs_dar_normaliser(n) == orc.dar_normaliser(n)
    assert G.gs_dar_normaliser(0) == 0.0


@pytest.mark.parametrize("field, value", [
    ("beta1", 1.0), ("beta2", -0.1), ("alpha1", 1.0), ("alpha2", -0.5), ("prec", 7), ("bias_mode", 2),
    ("reg_mode", 9), ("reserved", 1), ("n_pixels", 0), ("eps", float("nan")), ("lambda_o", float("inf")),
])
def test_init_rejects_bad_config_before_touching_device(G, field, value):
    cfg = G.make_config()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    s = G.lib().gs_opt_init(ctypes.byref(h), ctypes.byref(cfg), 10, None)
    assert s == G.GS_ERR_INVALID_ARG and not h.value


def test_init_rejects_bad_sizes_and_null(G):
    cfg = G.make_config()
    h = ctypes.c_void_p()
    assert G.lib().gs_opt_init(ctypes.byref(h), ctypes.byref(cfg), -1, None) == G.GS_ERR_INVALID_ARG
    assert G.lib().gs_opt_init(ctypes.byref(h), ctypes.byref(cfg), 2 ** 31, None) == G.GS_ERR_INVALID_ARG
    assert G.lib().gs_opt_init(None, ctypes.byref(cfg), 10, None) == G.GS_ERR_INVALID_ARG
    assert G.lib().gs_opt_init(ctypes.byref(h), None, 10, None) == G.GS_ERR_INVALID_ARG


def test_null_context_calls_are_rejected(G):
    L = G.lib()
    assert L.gs_opt_rows(None) == -1
    assert L.gs_bias_table_len(None) == -1
    assert L.gs_step(None, None, None, None, None, None) == G.GS_ERR_INVALID_ARG
    assert L.gs_reindex_state(None, None, None, 0, None) == G.GS_ERR_INVALID_ARG
    L.gs_opt_destroy(None)


def test_no_cpu_fallback_without_gpu(G):
    """A valid request on a machine without a usable GPU fails loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    s = G.lib().gs_opt_init(ctypes.byref(h), ctypes.byref(G.make_config()), 10, None)
    assert s != G.GS_OK and not h.value
