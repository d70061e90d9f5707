"""CPU checks of the C ABI: the library loads, exports every declared symbol,
its structs match the header, and host-only entry points behave (no GPU)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlmc.h")


@pytest.fixture(scope="module")
def m():
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as mod
    mod.lib()
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mlmc_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(m):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(m.LIB_PATH)
    bound = {s[0] for s in m.SIGNATURES}
    for name in names:
        assert hasattr(lib, name), name
        assert name in bound, name


def test_struct_layout_matches_header(m):
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "mlmc.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mlmc_config), offsetof(mlmc_config, seed),
             offsetof(mlmc_config, mg_omega), offsetof(mlmc_config, workspace_bytes),
             sizeof(mlmc_level_state), sizeof(mlmc_kernel_stat));
      return 0;
    }'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [ctypes.sizeof(m.Config), m.Config.seed.offset, m.Config.mg_omega.offset,
           m.Config.workspace_bytes.offset, ctypes.sizeof(m.LevelState),
           ctypes.sizeof(m.KernelStat)]
    assert [int(x) for x in out] == got


def test_host_only_entry_points(m):
    L = m.lib()
    cfg = m.config(dim=2, n_levels=4, coarse_cells=8)
    assert [L.mlmc_mesh_cells(ctypes.byref(cfg), k) for k in range(4)] == [8, 16, 32, 64]
    assert L.mlmc_mesh_cells(ctypes.byref(cfg), 4) == -1
    assert L.mlmc_level_cost(ctypes.byref(cfg), 0) == 49.0
    assert L.mlmc_level_cost(ctypes.byref(cfg), 1) == 225.0 + 49.0
    assert L.mlmc_node_stride(2, 16) == 320            # 17^2 = 289 -> 320
    assert L.mlmc_elem_stride(3, 4) == 64
    assert L.mlmc_node_stride(4, 16) == -1
    assert L.mlmc_status_str(m.MLMC_ERR_NOT_CONVERGED) == b"a solve hit max_iter"
    assert L.mlmc_kernel_count() > 10 and L.mlmc_kernel_name(0) == b"draw_xi"


@pytest.mark.parametrize("field,value", [("dim", 4), ("n_levels", 0), ("coarse_cells", 1),
                                         ("modes_per_dim", 0), ("sigma2", 0.0), ("rtol", 0.0),
                                         ("qoi", 7), ("solver", 9)])
def test_invalid_configs_rejected_before_any_device_call(m, field, value):
    cfg = m.config()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert m.lib().mlmc_plan_create(ctypes.byref(cfg), None, ctypes.byref(h)) == m.MLMC_ERR_INVALID
    assert not h.value


def test_gmg_and_box_validation(m):
    h = ctypes.c_void_p()
    cfg = m.config(solver="gmg", coarse_cells=12)       # GMG needs n0 = 2^k
    assert m.lib().mlmc_plan_create(ctypes.byref(cfg), None, ctypes.byref(h)) == m.MLMC_ERR_INVALID
    cfg = m.config(qoi="box", coarse_cells=6)           # 0.25 * 6 is not a node
    assert m.lib().mlmc_plan_create(ctypes.byref(cfg), None, ctypes.byref(h)) == m.MLMC_ERR_INVALID


def test_allocate_rejects_bad_input(m):
    import numpy as np
    V = np.array([1.0, -1.0])
    C = np.array([1.0, 2.0])
    N = np.zeros(2, dtype=np.int64)
    st = m.lib().mlmc_allocate(V.ctypes.data_as(m._DP), C.ctypes.data_as(m._DP), 2, 0.1,
                               N.ctypes.data_as(m._I64P))
    assert st == m.MLMC_ERR_INVALID
