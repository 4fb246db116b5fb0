"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/pp.h declares, the ctypes
structures match the C layout, and descriptor validation rejects bad input
before touching the device."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pp.h")


@pytest.fixture(scope="module")
def built():
    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as pp
    return pp


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(pp_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pp_init_grid", "pp_init_species", "pp_load_particles", "pp_step", "pp_deposit",
                 "pp_field_update", "pp_diagnostics"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = built.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in built.SIGNATURES, name


def test_ctypes_layout_matches_c(built, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "pp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(pp_grid_desc), offsetof(pp_grid_desc, stream),
         sizeof(pp_species_desc), sizeof(pp_diag), offsetof(pp_diag, n_slow), offsetof(pp_diag, relax_iters));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    import ctypes as C
    pp = built
    assert vals == [C.sizeof(pp.GridDesc), pp.GridDesc.stream.offset, C.sizeof(pp.SpeciesDesc),
                    C.sizeof(pp.Diag), pp.Diag.n_slow.offset, pp.Diag.relax_iters.offset]


@pytest.mark.parametrize("bad", [dict(dt=0.6), dict(field_order=5), dict(alpha=0.4), dict(shape_order=0),
                                 dict(n=(0, 8, 8)), dict(precision=3)])
def test_descriptor_validation_without_gpu(built, bad):
    kw = dict(n=(8, 8, 8), d=(0.5, 0.5, 0.5), dt=0.25)
    n = bad.pop("n", kw.pop("n"))
    dt = bad.pop("dt", kw.pop("dt"))
    with pytest.raises(built.PPError) as ei:
        built.Simulation(n, kw["d"], dt, stream=0, **bad)
    assert ei.value.code == built.PP_EINVAL


def test_batch_create_validation_without_gpu(built):
    import ctypes as C
    lib = built.lib()
    b = C.c_void_p()
    assert lib.pp_batch_create(C.byref(b), 0, 4) == built.PP_EINVAL
    assert lib.pp_batch_create(C.byref(b), 1 << 30, 0) == built.PP_EINVAL
    assert lib.pp_batch_create(C.byref(b), 1 << 30, 4) == built.PP_OK
    used = C.c_int64(-1)
    active = C.c_int(-1)
    assert lib.pp_batch_used(b, C.byref(used), C.byref(active)) == built.PP_OK
    assert (used.value, active.value) == (0, 0)
    state = C.c_int(-1)
    assert lib.pp_batch_poll(b, 0, None, C.byref(state)) == built.PP_OK and state.value == built.PP_BATCH_FREE
    assert lib.pp_batch_poll(b, 9, None, C.byref(state)) == built.PP_EINVAL
    assert lib.pp_batch_destroy(b) == built.PP_OK


def test_device_bytes_estimate_is_host_only_arithmetic():
    """pp_estimate_device_bytes needs no device: 21 padded mesh arrays (ghost
    width 6), FP64 rho and Gauss reference, per species two particle buffers
    of the rounded capacity, keys and permutation, per-key offsets and the
    sort counters (8 octant keys per tile-padded cell)."""
    import paper_1211_4575_gb300 as pp
    n, caps = (16, 24, 8), [1000, 0]
    got = pp.estimate_device_bytes(n, caps, pp.PP_MIXED32)
    padded = (16 + 12) * (24 + 12) * (8 + 12)
    cells = 16 * 24 * 8
    nkeys = 8 * 16 * 24 * 8
    rounded = [1024, 64]
    expect = padded * 4 * 21 + 16 * cells + sum(2 * 28 * c + 8 * c + 4 * (nkeys + 1) for c in rounded) + 4 * (nkeys + 1)
    assert got == expect
    # walls on x double the mesh along x; FP64 particles are 48 B and carry no permutation
    got64 = pp.estimate_device_bytes(n, [64], pp.PP_FP64, (pp.PP_BOUNDARY_WALLS, 0, 0))
    padded64 = (32 + 12) * (24 + 12) * (8 + 12)
    nk64 = 8 * 32 * 24 * 8
    assert got64 == padded64 * 8 * 21 + 16 * 32 * 24 * 8 + 2 * 48 * 64 + 4 * 64 + 4 * (nk64 + 1) + 4 * (nk64 + 1)
    assert pp.estimate_device_bytes(n, [-1]) == 0
