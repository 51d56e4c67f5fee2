"""The C ABI boundary without a GPU: the library builds and loads, exports every
function include/nlfem.h declares, and the binding's struct layouts match what a C
compiler makes of the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nlfem.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_10775_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (nl_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match():
    from paper_2005_10775_gb300 import nlfem
    for n in declared_functions():
        assert hasattr(nlfem, n), n


def test_struct_layouts_match_c(tmp_path):
    from paper_2005_10775_gb300 import nlfem
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "nlfem.h"
#define P(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f));
int main(void) {
    printf("nl_mesh %zu\\nnl_config %zu\\nnl_csr %zu\\nnl_batch_info %zu\\n", sizeof(nl_mesh), sizeof(nl_config),
           sizeof(nl_csr), sizeof(nl_batch_info));
    P(nl_mesh, elem_in_omega) P(nl_config, ngon_offsets) P(nl_config, cap_printed) P(nl_config, shifted)
    P(nl_config, prec) P(nl_csr, val) P(nl_csr, priv) P(nl_csr, n_qp_pairs)
    P(nl_batch_info, source) P(nl_batch_info, tuned_ms) P(nl_batch_info, default_ms)
    P(nl_batch_info, mode) P(nl_batch_info, streams)
    return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(got["nl_mesh"]) == ctypes.sizeof(nlfem.nl_mesh)
    assert int(got["nl_config"]) == ctypes.sizeof(nlfem.nl_config)
    assert int(got["nl_csr"]) == ctypes.sizeof(nlfem.nl_csr)
    assert int(got["nl_batch_info"]) == ctypes.sizeof(nlfem.nl_batch_info)
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert int(val) == getattr(getattr(nlfem, t), f).offset, key


def test_errors_without_gpu_are_reported_not_raised():
    # nl_create on a machine without a usable device returns a status, it does not abort
    from paper_2005_10775_gb300 import nlfem
    h = ctypes.c_void_p()
    st = nlfem.LIB.nl_create(ctypes.byref(h), 0, None)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        assert st == nlfem.NL_OK
        nlfem.LIB.nl_destroy(h)
    else:
        assert st == nlfem.NL_ECUDA


def test_binding_rejects_bad_vectors_before_any_launch():
    """The binding's in-place vectors are never cast or copied (a copy would lose the result):
    a float32 or short vector, a non-contiguous one, or a host array where nl_cg_noalloc needs
    device memory is rejected with NL_EINVAL before the library is called (no context and no
    GPU are needed to see it)."""
    torch = pytest.importorskip("torch")
    import numpy as np

    from paper_2005_10775_gb300 import nlfem as nl
    A = nl.nl_csr(n=10)
    ok = torch.zeros(10, dtype=torch.float64)
    bad = {"float32": torch.zeros(10, dtype=torch.float32), "short": torch.zeros(9, dtype=torch.float64),
           "strided": torch.zeros(20, dtype=torch.float64)[::2]}
    for name, v in bad.items():
        for b, x in ((v, ok), (ok, v)):
            with pytest.raises(nl.NlError) as e:
                nl.nl_cg_noalloc(None, A, b, x)
            assert e.value.status == nl.NL_EINVAL, name
    with pytest.raises(nl.NlError) as e:   # right shape and type, but host memory
        nl.nl_cg_noalloc(None, A, ok, ok.clone())
    assert e.value.status == nl.NL_EINVAL
    for x in (np.zeros(10, np.float32), np.zeros(11), np.zeros(20)[::2]):
        with pytest.raises(nl.NlError) as e:
            nl.nl_cg(None, A, np.zeros(10), x)
        assert e.value.status == nl.NL_EINVAL
    with pytest.raises(nl.NlError) as e:
        nl.nl_cg(None, A, np.zeros(7), np.zeros(10))
    assert e.value.status == nl.NL_EINVAL
