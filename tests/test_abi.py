"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/iqcc.h declares (CPU only: no kernel is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "iqcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iqcc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_08883_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("iqcc_load_hamiltonian", "iqcc_dress", "iqcc_prune", "iqcc_qmf_energy",
                     "iqcc_generator_abc", "iqcc_dis_gradients", "iqcc_iterate", "iqcc_export",
                     "iqcc_num_terms", "iqcc_get_stats", "iqcc_last_error", "iqcc_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_2603_08883_gb300 import iqcc
    assert set(_declared()) <= set(iqcc.exported_symbols())


def test_errors_without_a_device_are_reported_not_raised(lib):
    """With no GPU visible, creating a context fails with a status code and a
    message (no crash, no fallback)."""
    from paper_2603_08883_gb300 import iqcc
    import numpy as np
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is visible")
    except ImportError:
        pass
    with pytest.raises(iqcc.IqccError):
        iqcc.iqcc_load_hamiltonian(4, np.zeros((1, 1), np.uint64), np.zeros((1, 1), np.uint64), np.ones(1),
                                   use_torch=False)


def test_argument_errors_before_any_device_work(lib):
    from paper_2603_08883_gb300 import iqcc
    import numpy as np
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_load_hamiltonian(300, np.zeros((1, 5), np.uint64), np.zeros((1, 5), np.uint64), np.ones(1),
                                   use_torch=False)
    assert e.value.status == 1
    with pytest.raises(iqcc.IqccError) as e:   # a bit above n_qubits
        iqcc.iqcc_load_hamiltonian(3, np.array([[8]], np.uint64), np.zeros((1, 1), np.uint64), np.ones(1),
                                   use_torch=False)
    assert e.value.status == 1
    with pytest.raises(iqcc.IqccError) as e:   # index distances are stored in 8 bits
        iqcc.iqcc_load_hamiltonian(3, np.zeros((1, 1), np.uint64), np.zeros((1, 1), np.uint64), np.ones(1),
                                   max_probe=257, use_torch=False)
    assert e.value.status == 1


def test_ctypes_structs_match_the_header(tmp_path):
    """Size and field offsets of every struct the binding mirrors, as gcc lays
    them out from include/iqcc.h."""
    import subprocess
    from paper_2603_08883_gb300 import iqcc
    structs = {"iqcc_opts": iqcc.iqcc_opts, "iqcc_iter_opts": iqcc.iqcc_iter_opts,
               "iqcc_iter_result": iqcc.iqcc_iter_result, "iqcc_stats": iqcc.iqcc_stats,
               "iqcc_batch_screen_out": iqcc.iqcc_batch_screen_out, "iqcc_batch_info": iqcc.iqcc_batch_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{ROOT}/include/iqcc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            c_field = "free" if field == "free" else field
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {c_field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for line in out:
        if line:
            name, field, val = line.split()
            got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
