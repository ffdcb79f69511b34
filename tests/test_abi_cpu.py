"""Host-only checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every entry point include/apic.h declares, and validates configurations before
touching the device."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_1603_06188_gb300 import apic, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return apic.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "apic.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(apic_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("apic_create", "apic_p2g", "apic_grid_update", "apic_g2p", "apic_step", "apic_momentum"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    # and the binding mirrors the same names
    for name in declared_functions():
        assert hasattr(apic, name), name


def test_workspace_size_and_validation(lib):
    cfg = apic.make_config(dim=3, order=2, res=(128, 128, 128), dx=1 / 128)
    small = apic.apic_workspace_size(cfg, 1000)
    big = apic.apic_workspace_size(cfg, 4_000_000)
    assert 0 < small < big
    # cubic needs the same grid
    cfg3 = apic.make_config(dim=3, order=3, res=(128, 128, 128), dx=1 / 128)
    assert apic.apic_workspace_size(cfg3, 1000) > 0
    cases = [
        (dict(order=1), apic.APIC_ERR_UNSUPPORTED),      # multilinear: unstable B transfer (Sec. 5.9)
        (dict(order=4), apic.APIC_ERR_UNSUPPORTED),
        (dict(dim=4), apic.APIC_ERR_ARG),
        (dict(precision=16), apic.APIC_ERR_ARG),
        (dict(res=(3, 64, 64)), apic.APIC_ERR_ARG),
        (dict(res=(2048, 64, 64)), apic.APIC_ERR_ARG),
        (dict(dx=0.0), apic.APIC_ERR_ARG),
        (dict(tile_particles=100), apic.APIC_ERR_ARG),
        (dict(p2g_group=3), apic.APIC_ERR_ARG),
        (dict(p2g_kernel=9), apic.APIC_ERR_ARG),
        (dict(p2g_kernel=3), apic.APIC_ERR_ARG),
        (dict(dim=2, res=(64, 64), p2g_kernel=1), apic.APIC_ERR_ARG),   # component-split P2G is 3-D only
        (dict(model="fcr", E=-1.0, nu=0.3), apic.APIC_ERR_ARG),
        (dict(model="fcr", E=1.0, nu=0.5), apic.APIC_ERR_ARG),
    ]
    for kw, status in cases:
        base = dict(dim=3, order=2, res=(64, 64, 64), dx=1 / 64)
        base.update(kw)
        with pytest.raises(apic.ApicError) as e:
            apic.apic_workspace_size(apic.make_config(**base), 100)
        assert e.value.status == status, kw


def test_create_rejects_bad_workspace_without_touching_the_gpu(lib):
    cfg = apic.make_config(dim=3, order=2, res=(32, 32, 32), dx=1 / 32)
    with pytest.raises(apic.ApicError) as e:
        apic.apic_create(cfg, 10, 0, 0, 0)
    assert e.value.status == apic.APIC_ERR_ARG
    need = apic.apic_workspace_size(cfg, 10)
    with pytest.raises(apic.ApicError) as e:
        apic.apic_create(cfg, 10, 1 << 20, need - 1, 0)   # never dereferenced: size check comes first
    assert e.value.status == apic.APIC_ERR_OOM


@pytest.mark.parametrize("cname,pytype", [("apic_config", "Config"), ("apic_batch_config", "BatchConfig")])
def test_binding_structs_match_the_header(cname, pytype):
    """The ctypes mirrors of the configuration structs have the header's size and field
    offsets: a C program compiled against include/apic.h prints them."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    st = getattr(apic, pytype)
    lines = [f'printf("size %zu\\n", sizeof({cname}));']
    for name, _ in st._fields_:
        lines.append(f'printf("{name} %zu\\n", offsetof({cname}, {name}));')
    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"apic.h\"\nint main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c_path, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c_path, "w").write(src)
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), c_path, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    got = dict(zip(out[0::2], (int(v) for v in out[1::2])))
    assert got["size"] == ctypes.sizeof(st)
    for name, _ in st._fields_:
        assert got[name] == getattr(st, name).offset, name
