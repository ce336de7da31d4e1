"""The C-ABI library loads and exports every function include/katz.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(katz_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("katz_create_csr", "katz_rank_static", "katz_apply_update_batch", "katz_get_ranking",
                     "katz_get_bounds", "katz_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1807_03847_gb300 as K

    lib = ctypes.CDLL(K.library_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls():
    import paper_1807_03847_gb300 as K

    o = K.katz_default_opts()
    assert o.precision == K.KATZ_FP64 and o.undirected == 1 and o.r_max == 128
    assert K.katz_status_string(0) == "KATZ_OK" and K.katz_status_string(5) == "KATZ_ENOTCONV"


def test_struct_layout_matches_the_header(tmp_path):
    import subprocess
    import paper_1807_03847_gb300 as K

    src = tmp_path / "sz.c"
    src.write_text('#include "katz.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(katz_opts), sizeof(katz_info),'
                   ' offsetof(katz_opts, cuda_stream), offsetof(katz_info, affected), sizeof(katz_server_opts),'
                   ' sizeof(katz_request_result), offsetof(katz_request_result, latency_ms));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(K.katz_opts), ctypes.sizeof(K.katz_info), K.katz_opts.cuda_stream.offset,
                   K.katz_info.affected.offset, ctypes.sizeof(K.katz_server_opts),
                   ctypes.sizeof(K.katz_request_result), K.katz_request_result.latency_ms.offset]


def test_create_rejects_bad_arguments_without_touching_the_device():
    import numpy as np
    import paper_1807_03847_gb300 as K

    with pytest.raises(K.KatzError) as e:
        K.katz_create_csr(0, 0, np.zeros(1, np.int64), np.zeros(1, np.int32))
    assert e.value.name == "KATZ_EINVAL"


def test_server_options_are_checked_on_the_host():
    import paper_1807_03847_gb300 as K

    for kw in ({"admit_bytes": -1}, {"workers": 0}, {"slots": 0}, {"slot_updates": 0}):
        with pytest.raises(K.KatzError) as e:
            K.Server(**kw)
        assert e.value.name == "KATZ_EINVAL"
