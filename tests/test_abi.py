"""The C ABI library loads and exports every symbol include/melt.h declares
(no compute: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(melt_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt
    return melt


def test_header_declares_entry_points():
    names = _declared()
    for n in ["melt_basis_create", "melt_forward", "melt_destroy", "melt_basis_create_ex",
              "melt_sync", "melt_num_frames"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(so, n)]
    assert not missing, missing
    assert set(_declared()) <= set(lib.SIGNATURES), set(_declared()) - set(lib.SIGNATURES)


def test_host_only_calls(lib):
    assert lib.melt_version().startswith("melt")
    assert lib.melt_status_string(0) == "ok"
    assert lib.melt_status_string(-5) == "kernel wait timed out"
    assert lib.melt_num_frames(None, 16000) == 0
    assert lib.melt_num_outputs(None) == 0
    # without a device, creation reports it instead of crashing
    h = ctypes.c_void_p()
    st = lib.lib.melt_basis_create(16000.0, 400, 160, 80, 0.0, 8000.0, 0, ctypes.byref(h))
    import torch
    if not torch.cuda.is_available():
        assert st == lib.MELT_ERR_NO_DEVICE
    else:
        lib.melt_destroy(h)
    # argument checks come first
    assert lib.lib.melt_basis_create(16000.0, 400, 160, 0, 0.0, 8000.0, 0, ctypes.byref(h)) == lib.MELT_ERR_ARG
    assert lib.lib.melt_basis_create(16000.0, 400, 160, 80, 0.0, 9000.0, 0, ctypes.byref(h)) == lib.MELT_ERR_ARG
    assert lib.lib.melt_basis_create(16000.0, 400, 160, 80, 0.0, 8000.0, 0, None) == lib.MELT_ERR_ARG


def test_plan_struct_matches_binding(lib, tmp_path):
    """melt_plan in include/melt.h and the binding's MeltPlan agree field by field."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    fields = [f for f, _ in lib.MeltPlan._fields_]
    src = tmp_path / "plan_layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "melt.h"\n'
        "int main(void) {\n"
        '  printf("size %zu\\n", sizeof(melt_plan));\n'
        + "".join(f'  printf("{f} %zu\\n", offsetof(melt_plan, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "plan_layout"
    subprocess.run([cc, "-std=c99", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(lib.MeltPlan)
    for f in fields:
        assert int(got[f]) == getattr(lib.MeltPlan, f).offset, f


def test_padded_layout(lib):
    """Lengths, packed offsets and size of a batch after melt_pad_reflect: every
    padded clip starts on a 16-byte boundary, as melt_forward requires."""
    lens, offs, total = lib.padded_layout([201, 5, 4000], 200)
    assert lens.tolist() == [601, 405, 4400]
    assert offs.tolist() == [0, 604, 1012]
    assert total == 604 + 408 + 4400
    assert all(o % 4 == 0 for o in offs)
    lens, offs, total = lib.padded_layout([], 200)
    assert lens.size == 0 and total == 0


def test_pad_and_diag_argument_checks_need_no_device(lib):
    """melt_pad_reflect and melt_diag_wait_timeout reject bad arguments before any CUDA call."""
    import numpy as np
    L = lib.lib
    lens = np.array([10, 3], dtype=np.int64)
    lp = lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    buf = ctypes.c_void_p(16)  # never dereferenced: every case below fails its checks first
    assert L.melt_pad_reflect(buf, None, lp, 0, 2, buf, None, None) == lib.MELT_OK        # empty batch
    assert L.melt_pad_reflect(buf, None, None, 2, 2, buf, None, None) == lib.MELT_ERR_ARG  # no lengths
    assert L.melt_pad_reflect(buf, None, lp, 2, -1, buf, None, None) == lib.MELT_ERR_ARG   # negative pad
    assert L.melt_pad_reflect(buf, None, lp, 2, 3, buf, None, None) == lib.MELT_ERR_ARG    # clip of 3 <= pad
    assert L.melt_pad_reflect(None, None, lp, 2, 2, buf, None, None) == lib.MELT_ERR_ARG   # no input
    assert L.melt_diag_wait_timeout(None, None) == lib.MELT_ERR_ARG


def test_plain_c_consumer(lib, tmp_path):
    """A C99 program includes melt.h, links libmelt.so and calls host-only entry points."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "consumer.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "melt.h"
#include "melt_diag.h"
int main(void) {
  melt_basis* b = 0;
  if (strncmp(melt_version(), "melt", 4) != 0) return 1;
  if (strcmp(melt_status_string(MELT_ERR_TIMEOUT), "kernel wait timed out") != 0) return 2;
  if (melt_num_frames(0, 16000) != 0) return 3;
  if (melt_basis_create(16000.0, 400, 160, 0, 0.0, 8000.0, MELT_WIN_HANN_PERIODIC, &b) != MELT_ERR_ARG) return 4;
  if (melt_forward(0, 0, 0, 0, 1, 0, 0) != MELT_ERR_ARG) return 5;
  if (melt_diag_wait_timeout(0, 0) != MELT_ERR_ARG) return 6;
  printf("ok\n");
  return 0;
}
''')
    libdir = os.path.dirname(lib.LIB_PATH)
    exe = tmp_path / "consumer"
    subprocess.run([cc, "-std=c99", "-I", HEADER_DIR, str(src), "-o", str(exe), f"-L{libdir}", "-lmelt",
                    f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stderr)
