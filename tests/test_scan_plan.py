"""Host logic of the diagonal scan's kernel choice (pmcmc_scan_plan; no GPU needed): every plan
fits the look-back workspace pmcmc_scan reserves (a launch with more tiles than that is refused
with an invalid-argument error), covers the chain, follows the documented size boundaries, and
honours the environment overrides the scan reads."""
import ctypes as C
import os

import pytest

ENV_KEYS = ("PMCMC_SCAN_KERNEL", "PMCMC_SCAN_SHAPE", "PMCMC_SCAN_DCONST", "PMCMC_PIPE_CTAS",
            "PMCMC_SCAN_CLUSTER", "PMCMC_SCAN_SLOTS", "PMCMC_SCAN_LAG")


@pytest.fixture(scope="module")
def lib():
    from paper_2508_18413_gb300 import build, _lib
    return _lib.load(build.build())


@pytest.fixture
def env():
    """Set scan environment variables for one test; restores them afterwards."""
    saved = {k: os.environ.get(k) for k in ENV_KEYS}
    for k in ENV_KEYS:
        os.environ.pop(k, None)

    def set_(**kv):
        for k in ENV_KEYS:
            os.environ.pop(k, None)
        os.environ.update({k: str(v) for k, v in kv.items()})
    yield set_
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


KERNELS = ("rows", "rows_const_d", "register", "staged", "pipe", "cluster", "wide")
PREC = {"f64": 0, "f32": 1, "f32_scan_bf16": 2}


def plan(lib, precision, T, D):
    k, tile, tiles, mt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    st = lib.pmcmc_scan_plan(1, PREC[precision], T, D, C.byref(k), C.byref(tile), C.byref(tiles),
                             C.byref(mt))
    assert st == 0, (precision, T, D, st)
    return KERNELS[k.value], tile.value, tiles.value, mt.value


SIZES_T = [1, 7, 255, 4099, 100_003, 131_072, 262_145, 524_288, 1_000_003, 4_194_305, 33_554_432]
SIZES_D = [1, 2, 3, 4, 5, 8, 16, 18, 25, 32, 33, 64, 100, 256]
OVERRIDES = [{}, {"PMCMC_SCAN_KERNEL": "rows"}, {"PMCMC_SCAN_KERNEL": "staged"},
             {"PMCMC_SCAN_KERNEL": "pipe"}, {"PMCMC_SCAN_KERNEL": "pipe", "PMCMC_PIPE_CTAS": 2},
             {"PMCMC_SCAN_KERNEL": "cluster"},
             {"PMCMC_SCAN_KERNEL": "cluster", "PMCMC_SCAN_CLUSTER": 2, "PMCMC_SCAN_SLOTS": 8},
             {"PMCMC_SCAN_DCONST": 0}, {"PMCMC_SCAN_KERNEL": "rows", "PMCMC_SCAN_SHAPE": "16,5"},
             {"PMCMC_SCAN_KERNEL": "rows", "PMCMC_SCAN_SHAPE": "8,64"}]


@pytest.mark.parametrize("override", range(len(OVERRIDES)))
def test_every_plan_fits_the_workspace_and_covers_the_chain(lib, env, override):
    env(**OVERRIDES[override])
    for precision in PREC:
        for D in SIZES_D:
            for T in SIZES_T:
                if T * D > 2**31 // 8:
                    continue
                k, tile, tiles, mt = plan(lib, precision, T, D)
                assert tile > 0 and tiles * tile >= T > (tiles - 1) * tile, (precision, T, D, k)
                assert tiles <= mt, (precision, T, D, k, tiles, mt, OVERRIDES[override])


def test_default_choice_follows_the_size_boundaries(lib, env):
    env()
    D = 8
    for precision, hi in (("f32", 1 << 22), ("f32_scan_bf16", 3 << 21)):
        assert plan(lib, precision, ((1 << 20) - 8) // D, D)[0] in ("register", "rows_const_d")
        assert plan(lib, precision, (1 << 20) // D, D)[0] == "pipe"
        assert plan(lib, precision, hi // D, D)[0] == "pipe"
        assert plan(lib, precision, hi // D + 1, D)[0] == "rows_const_d"
        assert plan(lib, precision, (1 << 28) // D, D)[0] == "rows_const_d"
    # D not a power of two: the generic row kernel, pipelined for 2^21 < T D <= 3 2^22
    assert plan(lib, "f32", (1 << 21) // 32, 25)[0] in ("register", "rows")
    assert plan(lib, "f32", (1 << 21) // 25 + 1, 25)[0] == "pipe"
    assert plan(lib, "f32", (3 << 22) // 25 + 1, 25)[0] == "rows"
    # FP64 keeps the general boundaries
    assert plan(lib, "f64", (1 << 20) // D, D)[0] in ("register", "rows_const_d")
    assert plan(lib, "f64", (1 << 22) // D, D)[0] == "pipe"
    # wider states: the shared-memory kernel
    assert plan(lib, "f32", 10_000, 33)[0] == "wide"


def test_environment_overrides(lib, env):
    T, D = (1 << 26) // 8, 8
    env(PMCMC_SCAN_DCONST=0)
    assert plan(lib, "f32", T, D)[0] == "rows"
    env(PMCMC_SCAN_KERNEL="cluster")
    assert plan(lib, "f32", T, D)[0] == "cluster"
    assert plan(lib, "f32_scan_bf16", T, D)[0] == "cluster"
    assert plan(lib, "f64", T, D)[0] != "cluster"          # FP32 iterates only
    env(PMCMC_SCAN_KERNEL="rows", PMCMC_SCAN_SHAPE="16,5")
    k, tile, _, _ = plan(lib, "f32", T, D)
    assert k == "rows" and tile == 8 * 16 * 5 * (32 // D)
    env(PMCMC_SCAN_KERNEL="staged")
    assert plan(lib, "f32", T, D)[0] == "staged"


def test_invalid_arguments(lib):
    out = [C.c_int() for _ in range(4)]
    refs = [C.byref(o) for o in out]
    assert lib.pmcmc_scan_plan(1, 1, 0, 8, *refs) != 0          # T <= 0
    assert lib.pmcmc_scan_plan(1, 1, 100, 0, *refs) != 0        # D <= 0
    assert lib.pmcmc_scan_plan(1, 1, 100, 257, *refs) != 0      # D beyond the diagonal scan
    assert lib.pmcmc_scan_plan(0, 1, 100, 8, *refs) != 0        # dense: not planned here
    assert lib.pmcmc_scan_plan(1, 7, 100, 8, *refs) != 0        # unknown precision
    assert lib.pmcmc_scan_plan(1, 1, 100, 8, None, refs[1], refs[2], refs[3]) != 0
