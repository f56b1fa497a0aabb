"""C ABI checks that need no GPU: exports, struct layout, argument validation, sizes."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nufftjac.h")


@pytest.fixture(scope="module")
def abi():
    from paper_2111_02912_gb300 import _abi, build
    build.build()
    return _abi


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nufft_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_function(abi):
    declared = _declared_functions()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (nufft_\w+)", out))
    assert set(declared) == exported
    assert set(abi.EXPORTED) == exported
    lib = abi.lib()
    for name in declared:
        assert hasattr(lib, name)


def test_struct_layout_matches_c(abi, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "nufftjac.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(nufft_opts), offsetof(nufft_opts, sigma),'
                   ' offsetof(nufft_opts, bin_size), sizeof(nufft_plan_info), offsetof(nufft_plan_info, m),'
                   ' offsetof(nufft_plan_info, workspace_bytes)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(abi.nufft_opts), abi.nufft_opts.sigma.offset, abi.nufft_opts.bin_size.offset,
            ctypes.sizeof(abi.nufft_plan_info), abi.nufft_plan_info.m.offset,
            abi.nufft_plan_info.workspace_bytes.offset]
    assert got == want


def test_header_constants_match_the_binding(abi, tmp_path):
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "nufftjac.h"\n'
                   'int main(void){printf("%d %u %d %d\\n", NUFFT_MAX_COILS, NUFFT_NOALLOC_SCRATCH_BYTES,'
                   ' NUFFT_SPREAD_STRIPS, NUFFT_ERR_TIMEOUT); return 0;}\n')
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [abi.NUFFT_MAX_COILS, abi.NUFFT_NOALLOC_SCRATCH_BYTES, abi.NUFFT_SPREAD_STRIPS, abi.NUFFT_ERR_TIMEOUT]
    assert got == want


def test_default_opts_and_status_strings(abi):
    o = abi.nufft_default_opts(2, (320, 320))
    assert (o.dim, o.n[0], o.n[1], o.J, o.sigma, o.max_coils) == (2, 320, 320, 6, 2.0, 1)
    assert abi.status_string(0) == "ok"
    assert abi.status_string(-2) == "unsupported configuration"


@pytest.mark.parametrize("mutate,status", [
    (lambda o: setattr(o, "dim", 4), -2),
    (lambda o: o.n.__setitem__(0, 63), -2),
    (lambda o: setattr(o, "J", 9), -2),
    (lambda o: setattr(o, "sigma", 0.9), -2),
    (lambda o: setattr(o, "max_coils", 129), -2),   # NUFFT_MAX_COILS + 1
    (lambda o: o.n.__setitem__(0, 2), -2),          # K = 4 < J = 6
    (lambda o: o.n.__setitem__(1, 4000), -2),       # K = 8000 > 4096
])
def test_invalid_plans_are_rejected_before_touching_the_device(abi, mutate, status):
    o = abi.nufft_default_opts(2, (64, 64))
    mutate(o)
    with pytest.raises(abi.NufftError) as e:
        abi.nufft_plan(o, 0, None)
    assert e.value.status == status
    assert abi.nufft_workspace_bytes(o, 100, 0) == 0


def test_null_arguments(abi):
    lib = abi.lib()
    assert lib.nufft_plan(None, None, 0, None, None) == abi.NUFFT_ERR_INVALID_ARG
    assert lib.nufft_forward(None, 1, None, None, None, None) == abi.NUFFT_ERR_INVALID_ARG
    assert lib.nufft_set_points(None, 0, None, None) == abi.NUFFT_ERR_INVALID_ARG
    assert b"NULL" in lib.nufft_last_error()


def test_workspace_bytes_scale_with_coils_and_grid(abi):
    o = abi.nufft_default_opts(2, (320, 320))
    o.max_coils = 16
    b16 = abi.nufft_workspace_bytes(o, 51200)
    grid = 640 * 640 * 16 * 3 * 8
    # grids G and T, point records and sort tables, and for the strip spread the sorted coil values
    # (6.6 MB here), the hit lists (15 per point at most, 6.1 MB) and the partial sums (<= 16 MB)
    assert grid * 1.5 <= b16 <= grid * 1.5 + 40_000_000
    o.max_coils = 1
    assert abi.nufft_workspace_bytes(o, 51200) < b16 / 8
    assert abi.nufft_workspace_bytes(o, 51200, 16) == b16      # C overrides max_coils


def test_invalid_gather_variant_is_rejected(abi):
    o = abi.nufft_default_opts(2, (64, 64))
    o.gather_variant = 3
    with pytest.raises(abi.NufftError) as e:
        abi.nufft_plan(o, 0, None)
    assert e.value.status == abi.NUFFT_ERR_INVALID_ARG


@pytest.mark.parametrize("mode,density", [(2, 0), (-1, 0), (1, 8), (1, 70000)])
def test_invalid_kernel_mode_or_table_density_is_rejected(abi, mode, density):
    o = abi.nufft_default_opts(2, (64, 64))
    o.kernel_mode = mode
    o.table_density = density
    with pytest.raises(abi.NufftError) as e:
        abi.nufft_plan(o, 0, None)
    assert e.value.status == abi.NUFFT_ERR_INVALID_ARG
    assert abi.nufft_workspace_bytes(o, 100, 0) == 0


def test_table_mode_workspace_counts_the_table(abi):
    o = abi.nufft_default_opts(2, (64, 64))
    direct = abi.nufft_workspace_bytes(o, 1000, 1)
    o.kernel_mode = abi.NUFFT_KERNEL_TABLE
    o.table_density = 1024
    assert abi.nufft_workspace_bytes(o, 1000, 1) == direct + (1024 * 6 // 2 + 2) * 4


def test_largest_accepted_grids_and_first_refused(abi):
    """Size limits, checked on the host before the device is touched: the largest 2-D grid edge
    (K = 4096) with the most coils is accepted (its workspace is counted), one step past the edge is
    refused, and so are 3-D grids whose first-axis channel stride would overflow the 32-bit line
    offsets or whose bins overflow the point sort."""
    o = abi.nufft_default_opts(2, (2048, 2048))
    o.max_coils = abi.NUFFT_MAX_COILS
    assert abi.nufft_workspace_bytes(o, 1000, 0) > 3 * 4096 * 4096 * abi.NUFFT_MAX_COILS * 8
    for dim, n, coils, why in [(2, (2050, 2048), 1, "edge exceeds 4096"),
                               (3, (1024, 1024, 1024), abi.NUFFT_MAX_COILS, "too large for max_coils"),
                               (3, (1024, 1024, 1024), 1, "too large for the point sort")]:
        o = abi.nufft_default_opts(dim, n)
        o.max_coils = coils
        assert abi.nufft_workspace_bytes(o, 1000, 0) == 0
        with pytest.raises(abi.NufftError) as e:
            abi.nufft_plan(o, 0, None)
        assert e.value.status == abi.NUFFT_ERR_UNSUPPORTED and why in str(e.value)


@pytest.mark.parametrize("field,value,status,why", [
    ("beta", 200.0, -2, "beta too large"),
    ("spread_variant", 9, -1, "unknown spread_variant"),
    ("strip_part", 100, -1, "power of two"),
    ("strip_part", 8192, -1, "power of two"),
])
def test_invalid_spread_and_kernel_options_are_rejected(abi, field, value, status, why):
    o = abi.nufft_default_opts(2, (64, 64))
    setattr(o, field, value)
    assert abi.nufft_workspace_bytes(o, 100, 0) == 0
    with pytest.raises(abi.NufftError) as e:
        abi.nufft_plan(o, 0, None)
    assert e.value.status == status and why in str(e.value)


def test_deterministic_needs_the_strip_spread(abi):
    o = abi.nufft_default_opts(2, (64, 64))
    o.deterministic = 1
    o.spread_variant = abi.NUFFT_SPREAD_STRIPS
    assert abi.nufft_workspace_bytes(o, 100, 0) > 0
    o.strip_part = 4096                                  # the largest part size is accepted
    assert abi.nufft_workspace_bytes(o, 100, 0) > 0
    o.spread_variant = abi.NUFFT_SPREAD_TILES
    assert abi.nufft_workspace_bytes(o, 100, 0) == 0
    with pytest.raises(abi.NufftError) as e:
        abi.nufft_plan(o, 0, None)
    assert e.value.status == abi.NUFFT_ERR_UNSUPPORTED and "strip spread" in str(e.value)
