"""The C-ABI library builds, loads without a GPU, exports every entry point
that include/srm.h declares, matches the binding's struct layout, and
rejects bad arguments on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "srm.h")
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1608_04647_gb300 import _build, load_library
    _build.build()
    return load_library()


def declared_symbols():
    text = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"SRM_API\s+[\w\s\*]+?\b(srm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["srm_init", "srm_estep", "srm_mstep", "srm_fit", "srm_transform", "srm_get_w", "srm_get_s",
              "srm_get_params", "srm_get_state", "srm_set_state", "srm_last_error", "srm_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (srm_\w+)", out))
    for n in declared_symbols():
        assert n in exported, n
        assert hasattr(lib, n)


def test_config_struct_layout_matches_c(lib):
    from paper_1608_04647_gb300 import srm_config
    src = f'''#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(srm_config), offsetof(srm_config, n_subjects),
         offsetof(srm_config, voxels), offsetof(srm_config, T), offsetof(srm_config, k),
         offsetof(srm_config, in_dtype), offsetof(srm_config, store_dtype), offsetof(srm_config, flags),
         offsetof(srm_config, max_iter), offsetof(srm_config, seed));
  return 0;
}}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-o", exe, c], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    py = [ctypes.sizeof(srm_config)] + [getattr(srm_config, f).offset for f in
                                        ["n_subjects", "voxels", "T", "k", "in_dtype", "store_dtype", "flags",
                                         "max_iter", "seed"]]
    assert vals == py


def test_plan_struct_layout_matches_c(lib):
    """srm_plan: the binding's fields in the header's order, at the same offsets."""
    from paper_1608_04647_gb300 import srm_plan
    hdr = open(HEADER).read()
    head = hdr[:hdr.index("} srm_plan;")]
    body = head[head.rindex("typedef struct {"):]
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert fields == [n for n, _ in srm_plan._fields_]
    offs = ", ".join(f"offsetof(srm_plan, {f})" for f in fields)
    fmt = " ".join(["%zu"] * (len(fields) + 1))
    src = f'''#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("{fmt}\\n", sizeof(srm_plan), {offs});
  return 0;
}}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-o", exe, c], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(srm_plan)] + [getattr(srm_plan, f).offset for f in fields]


def test_plan_calls_reject_bad_arguments_without_a_gpu(lib):
    """The plan entry points check their arguments before any CUDA call."""
    from paper_1608_04647_gb300 import SRM_ERR_ARG, srm_plan
    p = srm_plan()
    assert lib.srm_get_plan(None, ctypes.byref(p)) == SRM_ERR_ARG
    assert lib.srm_set_plan(None, ctypes.byref(p)) == SRM_ERR_ARG
    assert lib.srm_autotune(None, None, 4, None, None, None, 0) == SRM_ERR_ARG


def _cfg(N=2, T=10, k=3, vox=(20, 30), store=0, flags=0):
    from paper_1608_04647_gb300 import srm_config
    arr = (ctypes.c_int64 * N)(*vox)
    cfg = srm_config(N, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64)), T, k, 0, store, flags, 0)
    cfg._keep = arr
    return cfg


@pytest.mark.parametrize("kw", [dict(k=0), dict(k=129), dict(T=1), dict(k=11, T=10), dict(vox=(2, 30)),
                                dict(store=1), dict(flags=1), dict(flags=1 << 20), dict(N=0, vox=())])
def test_host_side_argument_checks(lib, kw):
    from paper_1608_04647_gb300 import SRM_ERR_ARG
    cfg = _cfg(**kw)
    n = max(cfg.n_subjects, 1)
    dummy = (ctypes.c_void_p * n)(*([0x1000] * n))
    out = ctypes.c_void_p()
    st = lib.srm_init(ctypes.byref(cfg), dummy, dummy, None, ctypes.byref(out))
    assert st == SRM_ERR_ARG
    assert out.value is None
    assert lib.srm_last_error().decode().startswith("srm_init")


def test_null_arguments(lib):
    from paper_1608_04647_gb300 import SRM_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.srm_init(None, None, None, None, ctypes.byref(out)) == SRM_ERR_ARG
    cfg = _cfg()
    nulls = (ctypes.c_void_p * 2)(0x1000, 0)
    assert lib.srm_init(ctypes.byref(cfg), nulls, nulls, None, ctypes.byref(out)) == SRM_ERR_ARG
    for f in ("srm_estep", "srm_mstep", "srm_synchronize"):
        assert getattr(lib, f)(None) == SRM_ERR_ARG
    assert lib.srm_fit(None, 1, None) == SRM_ERR_ARG
    lib.srm_destroy(None)  # no-op


def test_flag_constants_match_header():
    import re

    import paper_1608_04647_gb300 as srm
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "srm.h")).read()
    defs = {m.group(1): 1 << int(m.group(2)) for m in re.finditer(r"#define (SRM_[A-Z_]+)\s+\(1u << (\d+)\)", hdr)}
    assert set(defs) >= {"SRM_BATCHED", "SRM_GRAPH", "SRM_FINAL_LL", "SRM_HOST_INPUT", "SRM_PROFILE",
                         "SRM_SINGLE_PASS"}
    for name, val in defs.items():
        assert getattr(srm, name) == val, name
