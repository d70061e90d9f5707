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
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def m():
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as mod
    mod.lib()
    return mod


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(mlmc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


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
    #include "mlmc_server.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mlmc_config), offsetof(mlmc_config, seed),
             offsetof(mlmc_config, mg_omega), offsetof(mlmc_config, workspace_bytes),
             sizeof(mlmc_level_state), sizeof(mlmc_kernel_stat), sizeof(mlmc_server_config),
             sizeof(mlmc_request_result), offsetof(mlmc_request_result, dof_solves),
             offsetof(mlmc_request_result, N));
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
           ctypes.sizeof(m.KernelStat), ctypes.sizeof(m.ServerConfig),
           ctypes.sizeof(m.RequestResult), m.RequestResult.dof_solves.offset,
           m.RequestResult.N.offset]
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


def test_server_entry_points_reject_bad_arguments_without_a_device(m):
    L = m.lib()
    h = ctypes.c_void_p()
    for sc in (m.ServerConfig(max_slots=0, pilot=8), m.ServerConfig(max_slots=4, pilot=1),
               m.ServerConfig(max_slots=1000, pilot=8), m.ServerConfig(max_slots=4, pilot=8, device=-1)):
        assert L.mlmc_server_create(ctypes.byref(sc), ctypes.byref(h)) == m.MLMC_ERR_INVALID
        assert not h.value
    cfg = m.config()
    rid = ctypes.c_uint64()
    assert L.mlmc_server_submit(None, ctypes.byref(cfg), 1e-3, ctypes.byref(rid)) == m.MLMC_ERR_INVALID
    done = ctypes.c_int()
    assert L.mlmc_server_poll(None, 1, ctypes.byref(done), None) == m.MLMC_ERR_INVALID
    assert L.mlmc_server_drain(None, 1.0) == m.MLMC_ERR_INVALID
    assert L.mlmc_server_clock(None) == -1.0
    assert L.mlmc_server_destroy(None) == m.MLMC_ERR_INVALID


def test_round_bytes_grows_with_counts(m):
    L = m.lib()
    cfg = m.config(dim=2, n_levels=3, coarse_cells=8, solver="gmg")
    arr = lambda xs: (ctypes.c_int64 * 3)(*xs)
    zero = L.mlmc_round_bytes(ctypes.byref(cfg), arr([0, 0, 0]))
    one = L.mlmc_round_bytes(ctypes.byref(cfg), arr([1, 1, 1]))
    two = L.mlmc_round_bytes(ctypes.byref(cfg), arr([2, 2, 2]))
    fine = L.mlmc_round_bytes(ctypes.byref(cfg), arr([0, 0, 4]))
    coarse = L.mlmc_round_bytes(ctypes.byref(cfg), arr([4, 0, 0]))
    assert zero == 0 and 0 < one < two and fine > coarse > 0
    cfg.dim = 7
    assert L.mlmc_round_bytes(ctypes.byref(cfg), arr([1, 1, 1])) == -1


def test_round_bytes_counts_the_nested_guess_buffer(m):
    """A coupled batch of level l > 0 keeps the coarse solution (one node
    array of mesh l-1 per sample) while the fine mesh is solved; level 0 has
    no coarse partner."""
    L = m.lib()
    arr = lambda xs: (ctypes.c_int64 * 3)(*xs)
    for dim, n0 in ((2, 8), (3, 4)):
        on = m.config(dim=dim, n_levels=3, coarse_cells=n0, solver="gmg", nested_guess=1)
        off = m.config(dim=dim, n_levels=3, coarse_cells=n0, solver="gmg", nested_guess=0)
        for level in range(3):
            for B in (1, 7, 64):
                counts = [0, 0, 0]
                counts[level] = B
                a = L.mlmc_round_bytes(ctypes.byref(on), arr(counts))
                b = L.mlmc_round_bytes(ctypes.byref(off), arr(counts))
                if level == 0:
                    assert a == b
                else:
                    guess = B * m.node_stride(dim, n0 << (level - 1)) * 8
                    assert guess <= a - b <= guess + 512
    bad = m.config(nested_guess=2)
    assert L.mlmc_round_bytes(ctypes.byref(bad), arr([1, 1, 1])) == -1


def test_kle_tensor_flag_validated_without_a_device(m):
    L = m.lib()
    assert m.config().kle_tensor == 0
    counts = (ctypes.c_int64 * 3)(1, 1, 1)
    ok = m.config(precision="mixed", kle_tensor=1)
    assert L.mlmc_round_bytes(ctypes.byref(ok), counts) > 0
    bad = m.config(precision="mixed", kle_tensor=2)
    assert L.mlmc_round_bytes(ctypes.byref(bad), counts) == -1
    assert L.mlmc_kappa32(None, 0, None, 1, None) == m.MLMC_ERR_INVALID


def test_stencil_tile_validated_without_a_device(m):
    L = m.lib()
    counts = (ctypes.c_int64 * 3)(1, 1, 1)
    for tile in (0, 1, 2):
        ok = m.config(dim=3, coarse_cells=8, precision="mixed", stencil_tile=tile)
        assert L.mlmc_round_bytes(ctypes.byref(ok), counts) > 0
    for tile in (-1, 3):
        bad = m.config(dim=3, coarse_cells=8, precision="mixed", stencil_tile=tile)
        assert L.mlmc_round_bytes(ctypes.byref(bad), counts) == -1


def test_coef_count_matches_the_oracle_mode_sets(m):
    from oracle import kle
    for dim, mpd, order in ((2, 8, -1), (3, 7, -1), (3, 16, 14), (2, 5, 3), (3, 4, 20)):
        cfg = m.config(dim=dim, modes_per_dim=mpd, total_order=order)
        assert m.coef_count(cfg) == kle.n_modes(dim, mpd, None if order < 0 else order)
    assert m.lib().mlmc_coef_count(ctypes.byref(m.config(dim=4))) == -1
