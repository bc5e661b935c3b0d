"""The C-ABI library loads and exports every function include/picmcc.h
declares; argument validation runs on the host (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "picmcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[\w ]+?\**\s*\b(\w+)\s*\(", src, flags=re.M))
    return {n for n in names if n.startswith(("pic_", "poisson_", "swarm_", "mlp_"))}


@pytest.fixture(scope="module")
def L():
    from paper_2110_14494_gb300 import build
    build.build()
    from paper_2110_14494_gb300 import picmcc
    return picmcc.lib()


def test_every_declared_symbol_is_exported(L):
    decl = _declared()
    assert len(decl) >= 19, decl
    for name in decl:
        assert hasattr(L, name), name
    from paper_2110_14494_gb300 import picmcc
    assert set(picmcc.EXPORTS) == decl


def test_status_strings(L):
    assert L.pic_status_string(0) == b"ok"
    assert L.pic_status_string(-3) == b"capacity exceeded"
    assert L.pic_status_string(7) == b"unknown status"


def test_host_argument_validation(L):
    import workloads as W
    from paper_2110_14494_gb300 import picmcc as P
    gas = P.Gas(W.synthetic_air())
    c = P.pic_config()
    c.precision, c.nx, c.ny, c.nz, c.dx, c.capacity, c.dt, c.gas = 32, 8, 8, 8, 1e-5, 1000, 1e-12, gas.c
    assert L.pic_workspace_bytes(C.byref(c)) > 0
    for field, bad in (("precision", 16), ("nx", 1), ("dx", 0.0), ("capacity", 0), ("dt", -1.0)):
        old = getattr(c, field)
        setattr(c, field, bad)
        assert L.pic_workspace_bytes(C.byref(c)) == 0, field
        setattr(c, field, old)
    h = C.c_void_p()
    assert L.pic_init(C.byref(c), None, 0, None, None, C.byref(h)) == P.PIC_ERR_ARG
    pc = P.poisson_config(1, 8, 8, 1e-5, 0, 0, 0)
    assert L.poisson_workspace_bytes(C.byref(pc)) == 0
    pc.nx = 8
    b64 = L.poisson_workspace_bytes(C.byref(pc))
    assert b64 > 0
    pc.precision = 32
    assert L.poisson_workspace_bytes(C.byref(pc)) > 0
    pc.precision = 16
    assert L.poisson_workspace_bytes(C.byref(pc)) == 0
    pc.precision = 0
    assert L.poisson_solve(C.byref(pc), None, None, None, None, None, None, 1e-6, 10, None, 0, None, None) == \
        P.PIC_ERR_ARG
    sc = P.swarm_config(64, gas.c, 2.45e25, 100, 10, 1000, 2000, 10, 1e-12, 1.0, 1, 0.25)
    assert L.swarm_workspace_bytes(C.byref(sc), 1) > 0
    sc.n_steps = 0
    assert L.swarm_workspace_bytes(C.byref(sc), 1) == 0


def test_mlp_host_validation(L):
    """Batch sizes the training kernels do not tile are refused on the host."""
    assert L.mlp_workspace_bytes(0) > 0
    assert L.mlp_workspace_bytes(4096) > L.mlp_workspace_bytes(0)
    for bad in (-1, 32, 100, 320):
        assert L.mlp_workspace_bytes(bad) == 0, bad
    from paper_2110_14494_gb300 import picmcc as P
    assert L.mlp_train(None, None, None, 0, None, None, 64, 1, 1e-3, 0.9, 0.999, 1e-8, None, None, 0, None) == \
        P.PIC_ERR_ARG
    assert L.mlp_forward(None, None, None, 10, None, 0, None) == P.PIC_ERR_ARG


def test_host_exchange_arrays_are_checked_before_the_call():
    """pic_upload / pic_download take raw host pointers: the binding refuses
    arrays of the wrong type, layout or length before the library sees them."""
    torch = pytest.importorskip("torch")
    from paper_2110_14494_gb300 import picmcc as P
    good32 = [np.zeros(100, np.float32) for _ in range(10)] + [np.zeros(100, np.int64)]
    assert len(P._host_arrays(good32, 100, 32, "t")) == 11
    good64 = [torch.zeros(100, dtype=torch.float64) for _ in range(10)] + [torch.zeros(100, dtype=torch.int64)]
    assert len(P._host_arrays(good64, 80, 64, "t")) == 11
    bad = [
        good32[:10],                                                          # 10 arrays
        [np.zeros(100, np.float64)] + good32[1:],                             # wrong precision
        good32[:10] + [np.zeros(100, np.int32)],                              # 32-bit ids
        good32[:3] + [np.zeros(99, np.float32)] + good32[4:],                 # too short
        good32[:5] + [np.zeros(200, np.float32)[::2]] + good32[6:],           # strided
        good32[:10] + [[0] * 100],                                            # not an array
        [torch.zeros(100, dtype=torch.float32)[::1].t() for _ in range(10)] + [torch.zeros(100, dtype=torch.int16)],
    ]
    for arrays in bad:
        with pytest.raises(ValueError):
            P._host_arrays(arrays, 100, 32, "t")


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the declaration in include/picmcc.h (a field added
    on one side only would shift the others)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import ctypes
    from paper_2110_14494_gb300 import picmcc as P
    names = [n for n in dir(P) if isinstance(getattr(P, n), type) and issubclass(getattr(P, n), ctypes.Structure)
             and n.startswith(("pic_", "poisson_", "swarm_"))]
    assert len(names) >= 9, names
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "picmcc.h"', "int main(void) {"]
    for s in names:
        src.append(f'printf("{s} . %zu\\n", sizeof({s}));')
        for f, _ in getattr(P, s)._fields_:
            src.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().split("\n"):
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for s in names:
        cls = getattr(P, s)
        assert got[(s, ".")] == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert got[(s, f)] == getattr(cls, f).offset, (s, f)


def test_noalloc_scratch_limit(L):
    """poisson_solve_noalloc works in a fixed 32 MiB device array: the
    workspace of a 96^3 solve fits in it and that of a 100^3 solve does not, at
    every precision (a change to the multigrid layout that moves the limit
    fails here)."""
    from paper_2110_14494_gb300 import picmcc as P
    for prec in (0, 32, 64):
        for n, fits in ((96, True), (100, False)):
            pc = P.poisson_config(n, n, n, 1e-5, 0.0, 1.0, 1.0, prec)
            b = L.poisson_workspace_bytes(C.byref(pc))
            assert b > 0 and (b <= 32 << 20) == fits, (prec, n, b)


def test_host_set_is_checked_once():
    """HostSet validates the 11 host arrays once (type, contiguity, capacity)
    for repeated pic_upload / pic_download calls."""
    from paper_2110_14494_gb300 import picmcc as P
    good = [np.zeros(100, np.float32) for _ in range(10)] + [np.zeros(100, np.int64)]
    hs = P.HostSet(good, 100, 32)
    assert hs.capacity == 100 and hs.precision == 32 and len(hs.ptrs) == 11
    with pytest.raises(ValueError):
        P.HostSet(good, 101, 32)   # arrays shorter than the capacity
    with pytest.raises(ValueError):
        P.HostSet(good, 100, 64)   # float32 arrays for a float64 set
