"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/cahn.h declares, the ctypes records match
the C layout, and argument validation answers before any CUDA call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1811_11842_gb300 import binding
from paper_1811_11842_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cahn.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return binding.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cahn_\w+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert "cahn_init" in names and "cahn_solve" in names
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(cahn_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(binding.SIGNATURES), "binding and header disagree"


def test_struct_layout_matches_header():
    fields = [f for f, _ in binding.cahn_params._fields_]
    sfields = [f for f, _ in binding.cahn_stats._fields_]
    src = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){",
           'printf("%zu\\n", sizeof(cahn_params));']
    src += [f'printf("%zu\\n", offsetof(cahn_params, {f}));' for f in fields]
    src += ['printf("%zu\\n", sizeof(cahn_stats));']
    src += [f'printf("%zu\\n", offsetof(cahn_stats, {f}));' for f in sfields]
    src += ["return 0;}"]
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write("\n".join(src))
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(binding.cahn_params)]
    want += [getattr(binding.cahn_params, f).offset for f in fields]
    want += [ctypes.sizeof(binding.cahn_stats)]
    want += [getattr(binding.cahn_stats, f).offset for f in sfields]
    assert vals == want


def test_nutrient_entry_points_reject_null_context(lib):
    assert lib.cahn_attach_nutrient(None, 0, None, None) == binding.CAHN_ERR_ARG
    assert lib.cahn_get_nutrient_history(None, 0, None) == binding.CAHN_ERR_ARG
    assert binding.cahn_tile_height(0, 0, binding.SYS_C, 0) == -1


def test_version_and_null_safety(lib):
    assert binding.cahn_abi_version() == 3
    assert lib.cahn_free(None) == 0
    assert lib.cahn_step(None, 1, None) == binding.CAHN_ERR_ARG
    assert isinstance(binding.cahn_last_error(None), str)


def _bad(prm_kw, lib):
    from paper_1811_11842_gb300 import inputs
    prm, _, _ = inputs.config_small()
    q = binding.make_params(prm.replace(**prm_kw))
    arr = (binding.cahn_params * 1)(q)
    fake = binding._ptr_array([16])      # never dereferenced: validation fails first
    ctx = ctypes.c_void_p()
    code = lib.cahn_init(ctypes.byref(ctx), 1, arr, fake, fake, fake, fake, None)
    return code, binding.cahn_last_error(None)


@pytest.mark.parametrize("kw,word", [
    (dict(nx=63), "nx"), (dict(ny=2), "ny"), (dict(dt=0.0), "dt"), (dict(eps=-1.0), "eps"),
    (dict(rho_biofilm=2.0), "densit"), (dict(restart=0), "restart"), (dict(rtol=2.0), "rtol"),
    (dict(max_iters=0), "max_iters"), (dict(flow_mode=7), "flow_mode"),
    (dict(nutrient=2), "nutrient"), (dict(nutrient=1, growth_kc=0.0), "growth_kc"),
    (dict(nutrient=1, diff_s=-1.0), "diff_s"), (dict(nutrient=1, consume_a=-1.0), "consume_a"),
    (dict(nutrient=1, c_bulk=float("nan")), "c_bulk"),
])
def test_invalid_params_rejected(lib, kw, word):
    code, msg = _bad(kw, lib)
    assert code == binding.CAHN_ERR_ARG
    assert word in msg


def test_invalid_batch_and_nulls(lib):
    ctx = ctypes.c_void_p()
    assert lib.cahn_init(ctypes.byref(ctx), 0, None, None, None, None, None, None) == binding.CAHN_ERR_ARG
    from paper_1811_11842_gb300 import inputs
    q = binding.make_params(inputs.config_small()[0])
    arr = (binding.cahn_params * 1)(q)
    nul = binding._ptr_array([0])
    assert lib.cahn_init(ctypes.byref(ctx), 1, arr, nul, nul, nul, nul, None) == binding.CAHN_ERR_ARG
    assert "NULL" in binding.cahn_last_error(None)


def test_make_params_marshals_every_field():
    """Every cahn_params field is taken from the Python record by name
    (the nutrient fields included)."""
    from paper_1811_11842_gb300 import inputs
    prm = inputs.config_nutrient()[0].replace(diff_s=1.7, growth_mu=0.3, growth_kc=0.2,
                                              growth_eps=0.9, consume_a=55.0, c_bulk=0.7,
                                              nutrient_bc=1, precond=1, use_graph=1)
    q = binding.make_params(prm)
    for name, _ in binding.cahn_params._fields_:
        assert getattr(q, name) == getattr(prm, name), name
