"""CPU-side checks of the C ABI: the library builds and loads, exports every
entry point that include/pic.h declares, its structs have the C layout, and the
host-side argument checks answer without touching a GPU."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")


@pytest.fixture(scope="module")
def P():
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def declared_functions():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(P):
    names = declared_functions()
    assert "pic_step" in names and "pic_create_grid" in names and len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pic_[a-z_0-9]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = P.library()
    for n in names:
        assert hasattr(lib, n)


def test_struct_layout_matches_c(P):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "pic.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(pic_grid_desc), offsetof(pic_grid_desc, precision),
         offsetof(pic_grid_desc, rho_bg), offsetof(pic_grid_desc, cuda_stream),
         sizeof(pic_diag), offsetof(pic_diag, n_particles));
  printf("%zu %zu\n", sizeof(pic_species_desc), offsetof(pic_grid_desc, sort_order));
  printf("%zu %zu %zu %zu\n", sizeof(pic_antenna_desc), offsetof(pic_antenna_desc, amplitude),
         offsetof(pic_antenna_desc, ramp), offsetof(pic_antenna_desc, start));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        with open(c, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    assert vals[0] == C.sizeof(P.pic_grid_desc)
    assert vals[1] == P.pic_grid_desc.precision.offset
    assert vals[2] == P.pic_grid_desc.rho_bg.offset
    assert vals[3] == P.pic_grid_desc.cuda_stream.offset
    assert vals[4] == C.sizeof(P.pic_diag)
    assert vals[5] == P.pic_diag.n_particles.offset
    assert vals[6] == C.sizeof(P.pic_species_desc)
    assert vals[7] == P.pic_grid_desc.sort_order.offset
    assert vals[8] == C.sizeof(P.pic_antenna_desc)
    assert vals[9] == P.pic_antenna_desc.amplitude.offset
    assert vals[10] == P.pic_antenna_desc.ramp.offset
    assert vals[11] == P.pic_antenna_desc.start.offset


def _create(P, **kw):
    args = dict(dims=2, n=(32, 32, 1), d=(1.0, 1.0, 1.0), dt=0.025, c=20.0)
    args.update(kw)
    desc = P.make_desc(args.pop("dims"), args.pop("n"), args.pop("d"), args.pop("dt"), args.pop("c"), **args)
    h = C.c_void_p()
    rc = P.library().pic_create_grid(C.byref(desc), C.byref(h))
    return rc, P.library().pic_last_error().decode()


def test_courant_limit_is_rejected_before_any_device_work(P):
    rc, msg = _create(P, dt=0.06, c=20.0)          # c dt / dx = 1.2
    assert rc == P.PIC_ERR_CFL and "Courant" in msg
    rc, msg = _create(P, dims=3, n=(32, 32, 32), dt=0.7, c=1.0)   # c dt sqrt(3) > 1
    assert rc == P.PIC_ERR_CFL and "Yee" in msg


@pytest.mark.parametrize("kw,code", [
    (dict(dims=4), 1), (dict(precision=7), 1),
    (dict(d=(0.0, 1.0, 1.0)), 1), (dict(halo=3), 1), (dict(n=(10, 32, 1)), 1),
])
def test_bad_descriptors_are_rejected(P, kw, code):
    rc, msg = _create(P, **kw)
    assert rc == code and msg


def test_2d_grid_needs_nz_1(P):
    desc = P.make_desc(2, (32, 32, 1), (1.0, 1.0, 1.0), 0.025, 20.0)
    desc.nz = 2
    h = C.c_void_p()
    assert P.library().pic_create_grid(C.byref(desc), C.byref(h)) == P.PIC_ERR_INVALID_ARG


def test_null_arguments_return_errors(P):
    lib = P.library()
    assert lib.pic_create_grid(None, None) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_step(None, 1) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_diagnostics(None, None) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_destroy(None) == P.PIC_OK
    assert lib.pic_num_particles(None, 0) == 0
    assert lib.pic_set_sort_policy(None, 1) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_set_adjoint_tiled(None, 1) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_step_saving(None, 1, None) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_state_restore(None, None, 0) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_state_restore_async(None, None, 0) == P.PIC_ERR_INVALID_ARG
    z = P._VP3()
    assert lib.pic_get_vector_potential(None, z, 0) == P.PIC_ERR_INVALID_ARG
    out = (C.c_double * 3)()
    assert lib.pic_generalized_momentum_run(None, 0, out) == P.PIC_ERR_INVALID_ARG
    z = P._VP3()
    assert lib.pic_adjoint_steps(None, None, 1, z, z, z, z) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_set_antenna(None, 0, None) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_renormalize_f32(None, None, C.c_longlong(5), None, None, None) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_renormalize_f32(None, None, C.c_longlong(-1), None, None, None) == P.PIC_ERR_INVALID_ARG
    assert lib.pic_measure_fp64_fma(C.c_longlong(0), 1, None, None, None) == P.PIC_ERR_INVALID_ARG
