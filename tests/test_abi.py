"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point declared in include/mmx.h, the
Python binding exposes the same names, descriptors are validated on the host,
and the product package never touches the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mmx.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mmx_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libmmx():
    from paper_2103_12819_b300 import _build
    path = _build.build()
    return ctypes.CDLL(path), path


def test_library_exports_every_declared_symbol(libmmx):
    L, path = libmmx
    names = _declared()
    assert len(names) >= 16
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mmx_\w+)", out))
    assert exported == set(names), (exported ^ set(names))


def test_binding_names_match_header():
    import paper_2103_12819_b300 as mmx
    assert sorted(mmx.EXPORTS) == _declared()


def test_library_is_built_for_sm103a_only():
    """The build passes exactly one -gencode, sm_103a code for compute_103a
    (no PTX for other architectures, no other SASS); the GPU test
    test_kernels_are_sm103_code checks the runtime's view of the binary."""
    from paper_2103_12819_b300 import _build
    flags = _build.NVCC_FLAGS
    gencodes = [flags[q + 1] for q, f in enumerate(flags) if f == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"], gencodes
    assert not any(f.startswith(("-arch", "--gpu-architecture", "-code")) for f in flags)


@pytest.mark.parametrize("bad", [
    dict(n=(0, 4, 4)), dict(dt=0.0), dict(order=3), dict(tol=0.0), dict(max_iter=0),
    dict(max_iter=65), dict(bc=(2, 1, 1)), dict(bc=(1, 1, 2), pml_cells=4), dict(prec=7),
])
def test_invalid_descriptors_rejected_on_host(bad):
    import paper_2103_12819_b300 as mmx
    kw = dict(n=(4, 4, 8), d=(1e-6,) * 3, dt=1e-15, bc=(1, 1, 1), pml_cells=0, order=2,
              tol=1e-10, max_iter=64, prec=0)
    kw.update(bad)
    with pytest.raises(mmx.MMXError) as ei:
        mmx.Solver(**kw)
    assert ei.value.code == -1


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2103_12819_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "mmx_oracle" not in text, f


def test_noalloc_rejects_grids_beyond_one_launch_row_per_z_node():
    """n = (7, 1, 65535): the padded size 8 * 2 * 65536 is exactly the scratch
    capacity, but its launch needs nz + 1 = 65536 grid rows along z, above
    the limit of 65535; the entry point refuses it on the host (no GPU call
    is made before the size checks)."""
    import paper_2103_12819_b300 as mmx
    n = (7, 1, 65535)
    count = (n[0] + 1) * n[1] * n[2]             # x-face extent
    rc = mmx.material_average_noalloc(n, (1, 1, 1), 3, 0x1000, 0x2000, count)
    assert rc == -1
