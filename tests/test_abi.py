"""The C-ABI library: it builds, loads and exports every symbol include/*.h declares;
argument validation on the host.  No GPU needed (no compute calls)."""
import ctypes as C
import glob
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_2511_06788_gb300.build import build
    build()
    import paper_2511_06788_gb300 as pkg
    return pkg.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(
            r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*((?:op|opnet)_[A-Za-z_0-9]*)\s*\(",
            src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("op_init", "op_step", "op_solve", "op_energy", "op_get_U",
                     "op_eigenvalues", "op_destroy", "op_apply_H", "op_gram", "op_core",
                     "op_update", "op_cg_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_2511_06788_gb300 import binding
    src = open(binding.__file__).read()
    missing = [n for n in declared_functions() if f'"{n}"' not in src]
    assert not missing, missing


def test_header_declares_the_network_api():
    names = declared_functions()
    for required in ("opnet_create", "opnet_forward", "opnet_infer", "opnet_loss_grad",
                     "opnet_train_step", "opnet_conv", "opnet_conv_dgrad", "opnet_destroy"):
        assert required in names


STRUCTS = {
    # C struct -> (binding class name, fields)
    "op_problem": ("OpProblem", ["dim", "shape", "lo", "hi", "p", "sigma", "tau", "prec",
                                 "cg_rtol", "cg_max_iter", "check_every", "adapt_every",
                                 "cg_precond", "flow", "fp64_gemm", "step1"]),
    "op_stats": ("OpStats", ["steps", "last_cg_iters", "cg_iters", "energy", "err_E",
                             "residual", "g_residual", "orth", "sigma", "tau", "ms"]),
    "op_shard_stats": ("OpShardStats", ["slabs", "halo_copies", "halo_bytes", "reductions",
                                        "reduction_bytes"]),
    "opnet_config": ("OpnetConfig", ["N", "lo", "hi", "p", "width", "stream"]),
}


def test_binding_structs_match_the_header_layout(tmp_path):
    """sizeof and offsetof of every struct the binding mirrors, from the C compiler on the
    headers themselves, equal the ctypes layout (a field added to one side only fails)."""
    import shutil
    import subprocess
    from paper_2511_06788_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "opevo.h"',
             '#include "opnet.h"', "int main(void) {"]
    for st, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        st, key, val = line.split()
        got[(st, key)] = int(val)
    for st, (cls_name, fields) in STRUCTS.items():
        cls = getattr(binding, cls_name)
        assert [f for f, _ in cls._fields_] == fields, st
        assert C.sizeof(cls) == got[(st, "size")], st
        for f in fields:
            assert getattr(cls, f).offset == got[(st, f)], (st, f)


def test_version_string(lib):
    assert b"sm_103a" in lib.op_version()


def _init_status(pb, V, U0):
    from paper_2511_06788_gb300 import binding as b
    ctx = C.c_void_p()
    s = b.lib().op_init(C.byref(ctx), C.byref(pb), V, U0, C.c_void_p(0))
    return s, ctx, b.last_error()


@pytest.mark.parametrize("bad", ["dim", "p0", "shape", "box", "prec", "precond", "flow",
                                 "l2_adapt", "l2_wide", "null"])
def test_init_rejects_bad_arguments_before_any_device_work(lib, bad):
    from paper_2511_06788_gb300 import binding as b
    pb = b.make_problem((4, 4), (0, 0), (1, 1), 2)
    V = np.zeros(16)
    U0 = np.ones((16, 2))
    Vp, Up = V.ctypes.data_as(C.POINTER(C.c_double)), U0.ctypes.data_as(C.POINTER(C.c_double))
    if bad == "dim":
        pb.dim = 4
    elif bad == "p0":
        pb.p = 0
    elif bad == "shape":
        pb.shape[1] = 0
    elif bad == "box":
        pb.hi[0] = pb.lo[0]
    elif bad == "prec":
        pb.prec = 9
    elif bad == "precond":
        pb.cg_precond = 2
    elif bad == "flow":
        pb.flow = 2
    elif bad == "l2_adapt":
        pb.flow, pb.adapt_every = 1, 10
    elif bad == "l2_wide":  # the exact Cayley step of the L2 flow takes p <= 256
        pb = b.make_problem((20, 20), (0, 0), (1, 1), 257, flow="l2")
        V, U0 = np.zeros(400), np.ones((400, 257))
        Vp = V.ctypes.data_as(C.POINTER(C.c_double))
        Up = U0.ctypes.data_as(C.POINTER(C.c_double))
    elif bad == "null":
        Vp = None
    s, ctx, msg = _init_status(pb, Vp, Up)
    assert s == b.OP_ERR_ARG and not ctx.value and msg


def test_p_larger_than_grid_rejected(lib):
    from paper_2511_06788_gb300 import binding as b
    pb = b.make_problem((2, 2), (0, 0), (1, 1), 5)
    V, U0 = np.zeros(4), np.ones((4, 5))
    s, _, msg = _init_status(pb, V.ctypes.data_as(C.POINTER(C.c_double)),
                             U0.ctypes.data_as(C.POINTER(C.c_double)))
    assert s == b.OP_ERR_ARG and "exceeds" in msg


def test_kernel_level_argument_checks(lib):
    from paper_2511_06788_gb300 import binding as b
    L = b.lib()
    # ld not a multiple of 8
    assert L.op_update(b.OP_FP64, 10, 3, 6, C.c_void_p(16), C.c_void_p(32), C.c_void_p(48),
                       C.c_void_p(64), C.c_void_p(80), C.c_void_p(96), 1 << 20,
                       C.c_void_p(0)) == b.OP_ERR_ARG
    # misaligned pointer
    assert L.op_gram(b.OP_FP32, 10, 3, 8, C.c_void_p(17), C.c_void_p(32), None, None, None,
                     None, 0, C.c_void_p(0)) == b.OP_ERR_ARG
    # non-positive tau in the core
    assert L.op_core(b.OP_FP64, 3, 8, -1.0, C.c_void_p(16), C.c_void_p(32), C.c_void_p(48),
                     C.c_void_p(64), None, None, C.c_void_p(128), 1 << 20,
                     C.c_void_p(0)) == b.OP_ERR_ARG
    # workspace queries are host-only arithmetic
    assert L.op_gram_workspace(b.OP_FP32, 1000, 64) > 0
    pb = b.make_problem((8, 8, 8), (0, 0, 0), (1, 1, 1), 16)
    assert L.op_cg_workspace(C.byref(pb), 16) >= 3 * 512 * 16 * 8


def test_problem_defaults_match_oracle_readings():
    """The NaN defaults of op_problem (sigma, tau) follow the oracle's readings."""
    import oracle as o
    import synthetic as syn
    P = syn.config_3d_wells(0, 16, 8)
    L = o.spectrum_lower_bound(P.shape, P.lo, P.hi, P.V)
    assert o.default_sigma(P.shape, P.lo, P.hi, P.V) == pytest.approx(max(0.0, 1 - L))
    assert math.isfinite(L)
