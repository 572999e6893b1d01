"""CPU checks of the C ABI library: it builds, loads without a GPU, and exports
every function that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            before = text[:m.start()].rstrip()
            # a declaration: preceded by a return type token, not a keyword/macro use
            if name in ("if", "sizeof", "defined") or before.endswith(("#define", "#if")):
                continue
            if re.search(r"(kf_status|void|const char\s*\*|int64_t|int32_t)\s*\**\s*$", before):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_1107_4192_gb300 import build
    return build.build()


def test_headers_declare_the_interface():
    names = declared_functions()
    for required in ("kf_plan", "kf_filter", "fis_smooth", "mne_solve", "kf_plan_destroy", "kf_strerror"):
        assert required in names


def test_library_loads_and_exports_all_declared(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/*.h but not exported"


def test_binding_signatures_cover_headers(built_lib):
    from paper_1107_4192_gb300 import binding
    assert set(declared_functions()) == set(binding.exported_symbols())


def test_strerror_host_only(built_lib):
    from paper_1107_4192_gb300 import binding
    assert binding.strerror(0) == "ok"
    assert "positive definite" in binding.strerror(binding.KF_ERR_NOT_PD)


def test_footprint_and_checkpoint_policy(built_lib):
    """Host-only sizing: full store when it fits, checkpoints when over budget, BUDGET when hopeless."""
    from paper_1107_4192_gb300 import binding as B
    d = B.make_desc(8196, 306, 300, prec=B.KF_PREC_MIXED_BF16X3, solve_prec=B.KF_SOLVE_FP32, stream=0)
    st, w, s, c = B.kf_plan_footprint(d)
    assert st == 0 and c == 1
    ldN = 8320
    assert s == 301 * 8196 * ldN * 4
    d.mem_budget_bytes = w + 40 * 8196 * ldN * 4
    st, w2, s2, c2 = B.kf_plan_footprint(d)
    assert st == 0 and c2 > 1 and w2 + s2 <= d.mem_budget_bytes
    assert s2 == (300 // c2 + 1 + 1 + c2 - 1) * 8196 * ldN * 4
    d.mem_budget_bytes = w + 5 * 8196 * ldN * 4
    st, *_ = B.kf_plan_footprint(d)
    assert st == B.KF_ERR_BUDGET


def test_footprint_rejects_bad_descriptors(built_lib):
    from paper_1107_4192_gb300 import binding as B
    for kw in (dict(N=0), dict(m=0), dict(T=0)):
        args = dict(N=10, m=3, T=4)
        args.update(kw)
        d = B.make_desc(args["N"], args["m"], args["T"], stream=0)
        assert B.kf_plan_footprint(d)[0] == B.KF_ERR_ARG
    d = B.make_desc(10, 3, 4, f_kind=B.KF_F_CSR, f_nnz=0, stream=0)
    assert B.kf_plan_footprint(d)[0] == B.KF_ERR_ARG
    d = B.make_desc(10, 3, 4, q_kind=7, stream=0)
    assert B.kf_plan_footprint(d)[0] == B.KF_ERR_ARG
