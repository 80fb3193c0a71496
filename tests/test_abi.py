"""The C-ABI library builds for sm_103a, loads, and exports every function include/helm.h declares
(no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2602_07711_gb300 import build as b
    if not os.path.exists(b.LIB) or any(os.path.getmtime(s) > os.path.getmtime(b.LIB) for s in b.sources()):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("helm_setup", "helm_apply_A", "helm_apply_precond", "helm_gmres_solve", "helm_build_rhs", "helm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(L, n), n


def test_status_strings_and_version(libpath):
    from paper_2602_07711_gb300 import helm
    L = helm.lib()
    assert L.helm_version().startswith(b"helm-gb300")
    for code in range(11):
        assert L.helm_status_str(code) and L.helm_status_str(code) != b"unknown status"


def test_setup_rejects_bad_arguments_without_gpu_work(libpath):
    from paper_2602_07711_gb300 import helm
    import numpy as np
    L = helm.lib()
    ctx = ctypes.c_void_p()
    g = helm.helm_grid(2, 8, 8, 1.0, 1.0, 1.0, 1)        # N < 4 is rejected before any CUDA call
    o = helm.helm_options(4, 1, 0, 30, 100, 1e-6, 0, 0)
    k2 = np.zeros(2 * 8 * 8, np.complex128)
    assert L.helm_setup(ctypes.byref(g), k2.ctypes.data, 1.0, None, ctypes.byref(o), None, ctypes.byref(ctx)) == 1
    g = helm.helm_grid(8, 8, 8, 1.0, 1.0, 1.0, 1)
    o = helm.helm_options(5, 1, 0, 30, 100, 1e-6, 0, 0)    # order 5 does not exist
    k2 = np.zeros(512, np.complex128)
    assert L.helm_setup(ctypes.byref(g), k2.ctypes.data, 1.0, None, ctypes.byref(o), None, ctypes.byref(ctx)) == 1
    assert L.helm_setup(None, None, 1.0, None, None, None, ctypes.byref(ctx)) == 1


def test_setup_checks_the_precision_and_the_wait_limit_without_gpu_work(libpath):
    """HELM_PREC_FP32, _TF32, _TF32X3 (the three-product split), _BF16 and _FP16 are the arithmetic modes; anything
    else is rejected before any device work, as is a wait limit without a context or below zero."""
    from paper_2602_07711_gb300 import helm
    import numpy as np
    L = helm.lib()
    ctx = ctypes.c_void_p()
    g = helm.helm_grid(8, 8, 8, 1.0, 1.0, 1.0, 0)
    k2 = np.zeros(512, np.complex128)
    assert (helm.HELM_PREC_FP32, helm.HELM_PREC_TF32, helm.HELM_PREC_TF32X3, helm.HELM_PREC_BF16,
            helm.HELM_PREC_FP16) == (0, 1, 2, 3, 4)
    for precision in (-1, 5):
        o = helm.helm_options(4, helm.HELM_PRECOND_PFFT, precision, 30, 100, 1e-6, 1, 0)
        assert L.helm_setup(ctypes.byref(g), k2.ctypes.data, 1.0, None, ctypes.byref(o), None,
                            ctypes.byref(ctx)) == 1
        assert not ctx.value
    assert L.helm_set_wait_limit(None, 5) == 1
    assert L.helm_set_matvec_variant(None, 0) == 1


def test_closure_entry_points_reject_null_contexts_without_gpu_work(libpath):
    from paper_2602_07711_gb300 import helm
    L = helm.lib()
    assert L.helm_set_closure(None, helm.HELM_CLOSURE_HIGH_ORDER) == 1
    assert L.helm_closure_face_count(None) == 0
    assert L.helm_build_rhs_fields(None, None, None, None) == 1
    assert L.helm_closure_rhs(None, None, None, None, None) == 1


def test_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    """Without libhelm.so every entry point raises: there is no CPU or other fallback on the product path."""
    import numpy as np

    from paper_2602_07711_gb300 import helm
    monkeypatch.setattr(helm, "library_path", str(tmp_path / "libhelm.so"))
    monkeypatch.setattr(helm, "_lib", None)
    with pytest.raises(RuntimeError, match="libhelm.so not found"):
        helm.lib()
    with pytest.raises(RuntimeError, match="libhelm.so not found"):
        helm.Solver((8, 8, 8), np.ones((8, 8, 8), complex), 1.0, order=4)


def test_header_is_c99_and_a_c_program_links_and_calls_the_library(libpath, tmp_path):
    """include/helm.h compiles as strict C99 and a C program links against libhelm.so and calls it (only
    entry points that do no GPU work: the version, status strings, and a rejected set-up)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "helm.h"
int main(void) {
    helm_ctx* ctx = (helm_ctx*)&ctx;
    helm_status st = helm_setup(NULL, NULL, 1.0, NULL, NULL, NULL, &ctx);
    if (st != HELM_ERR_ARG || ctx != NULL) return 2;
    if (strncmp(helm_version(), "helm-gb300", 10) != 0) return 3;
    if (strcmp(helm_status_str(HELM_OK), helm_status_str(HELM_ERR_ARG)) == 0) return 4;
    printf("%s\n", helm_status_str(st));
    return 0;
}
''')
    exe = tmp_path / "abi"
    libdir = os.path.dirname(libpath)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lhelm", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip()


def test_every_entry_point_rejects_a_null_context_without_gpu_work(libpath):
    """A NULL context (or net, or batch) is HELM_ERR_ARG for every call that takes one, constructors given
    bad arguments return HELM_ERR_ARG with *out = NULL, size queries return 0 and destroy(NULL) is a no-op."""
    from paper_2602_07711_gb300 import helm
    C = ctypes
    L = helm.lib()
    skip = {"helm_net_create", "helm_batch_create", "helm_gmres_solve_batched", "helm_setup", "helm_autotune"}
    checked = 0
    for name, (rt, args) in helm._SIGS.items():
        if rt is not C.c_int or not args or args[0] is not C.c_void_p or name in skip:
            continue
        vals = [0 if a in (C.c_int, C.c_uint, C.c_longlong, C.c_size_t) else 0.0 if a in (C.c_float, C.c_double)
                else None for a in args]
        assert getattr(L, name)(*vals) == 1, name
        checked += 1
    assert checked >= 25
    h = C.c_void_p(1)
    assert L.helm_net_create(0, 0, C.byref(h)) == 1 and h.value is None
    assert L.helm_net_create(8, 0, None) == 1
    h = C.c_void_p(1)
    assert L.helm_batch_create(None, 0, None, None, 0, None, C.byref(h)) == 1 and h.value is None
    assert L.helm_gmres_solve_batched(None, 0, None, None, 0, None, None) == 1
    assert L.helm_autotune(None, None, None, None, None) == 1
    assert L.helm_closure_face_count(None) == 0 and L.helm_net_num_params(None) == 0
    L.helm_destroy(None)
    L.helm_batch_destroy(None)
    L.helm_net_destroy(None)


def test_setup_rejects_grids_of_2_to_the_31_points_without_gpu_work(libpath):
    from paper_2602_07711_gb300 import helm
    import numpy as np
    L = helm.lib()
    ctx = ctypes.c_void_p(1)
    g = helm.helm_grid(4096, 4096, 128, 1.0, 1.0, 1.0, 1)   # 2^31 points: rejected before any CUDA call
    o = helm.helm_options(4, 1, 0, 30, 100, 1e-6, 0, 0)
    k2 = np.zeros(8, np.complex128)                          # not read
    assert L.helm_setup(ctypes.byref(g), k2.ctypes.data, 1.0, None, ctypes.byref(o), None, ctypes.byref(ctx)) == 10
    assert ctx.value is None
