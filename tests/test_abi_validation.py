"""Argument checking of every C-ABI entry point, on the CPU: an invalid
argument i (1-based) returns -i before anything is enqueued, as include/cf.h
states.  Each case starts from a valid-looking call (fake, aligned device
addresses that are never dereferenced: the checks run first) and breaks one
argument; the arguments before it stay valid, so the first check that fails
is that argument's own."""
import ctypes

import pytest

from paper_2108_09337_gb300 import cf

L = cf.lib()
P = 0x100000          # a fake, 1 MiB-aligned device address
BIG = 1 << 40         # any workspace size


def _opt(**kw):
    return ctypes.byref(cf.options(**kw))


# name: (valid-looking arguments, [(1-based position, invalid value), ...])
CASES = {
    "cf_tourn_select": ((100, 8, P, 100, 16, 2, P, P, BIG, None),
                        [(1, -1), (2, -1), (2, 129), (3, None), (4, 99), (5, 0), (5, 129), (6, 1), (6, 9), (7, None)]),
    "cf_tourn_select_f32": ((100, 8, P, 100, 16, 2, P, P, BIG, None),
                            [(1, -1), (2, 129), (3, None), (4, 99), (5, 0), (5, 513), (6, 1), (6, 9), (7, None)]),
    "cf_getrf": ((8, P, 8, P, P, P, BIG, None, None),
                 [(1, -1), (2, None), (3, 7), (4, None), (5, None)]),
    "cf_getrf_noalloc": ((8, P, 8, P, P, None, None),
                         [(1, -1), (2, None), (3, 7), (4, None), (5, None)]),
    "cf_potrf": ((8, P, 8, P, P, BIG, None, None),
                 [(1, -1), (2, None), (3, 7), (4, None)]),
    "cf_getrs": ((8, 2, P, 8, P, P, 8, P, BIG, None),
                 [(1, -1), (2, -1), (3, None), (4, 7), (5, None), (6, None), (7, 7)]),
    "cf_potrs": ((8, 2, P, 8, P, 8, None),
                 [(1, -1), (2, -1), (3, None), (4, 7), (5, None), (6, 7)]),
    "cf_residual": ((8, 6, 2, P, 8, P, 6, P, 8, P, 8, None),
                    [(1, -1), (2, -1), (3, -1), (4, None), (5, 7), (6, None), (7, 5), (8, None), (9, 7),
                     (10, None), (11, 7)]),
    "cf_residual_pair": ((8, 6, 2, P, 8, P, 6, P, 8, P, 8, P, BIG, None),
                         [(1, -1), (2, -1), (3, -1), (4, None), (5, 7), (6, None), (7, 5), (8, None), (9, 7),
                          (10, None), (11, 7)]),
    "cf_schur_update_lp": ((256, 256, 128, P, 128, P, 128, P, 256, 2, 0, None),
                           [(1, -1), (2, -1), (3, -64), (3, 100), (4, None), (5, 64), (5, 132), (6, None),
                            (7, 64), (7, 130), (8, None), (9, 255), (10, 0), (10, 4)]),
    "cf_schur_update_lp_splitk": ((256, 256, 128, P, 128, P, 128, P, 256, 2, 0, 2, P, BIG, None),
                                  [(1, -1), (2, -1), (3, -64), (3, 100), (4, None), (5, 64), (6, None), (7, 64),
                                   (8, None), (9, 255), (10, 0), (12, 0), (12, 65)]),
    "cf_quantize_e4m3": ((256, 200, P, 256, P, 256, P, 2, None),
                         [(1, -1), (2, -1), (3, None), (4, 255), (5, None), (6, 128), (6, 264), (7, None),
                          (8, 1)]),
    "cf_schur_update_fp8": ((256, 256, 256, P, 256, P, 2, P, 256, P, 2, P, 256, 0, None),
                            [(1, -1), (2, -1), (3, 100), (4, None), (5, 128), (5, 264), (6, None), (7, 1),
                             (8, None), (9, 128), (10, None), (11, 1), (12, None), (13, 255)]),
    "cf_factor_batched": ((4, None, 0, P, P, P, P, P, P, BIG, None, None),
                          [(1, -1), (3, 2), (4, None), (5, None), (6, None), (7, None), (8, None)]),
    "cf_getrf_batched": ((4, P, P, P, P, P, P, BIG, None, None),
                         [(1, -1), (2, None), (3, None), (4, None), (5, None), (6, None)]),
    "cf_potrf_batched": ((4, P, P, P, P, P, BIG, None, None),
                         [(1, -1), (2, None), (3, None), (4, None), (5, None)]),
    "cf_solve_batched_mixed": ((4, None, 0, P, P, P, P, P, P, P, P, None, P, BIG, None, None),
                               [(1, -1), (3, 5), (4, None), (5, None), (6, None), (7, None), (8, None),
                                (9, None), (10, None), (11, None)]),
    "cf_gesv_mixed": ((8, 2, P, 8, P, 8, P, 8, 3, P, None, P, BIG, None, None),
                      [(1, -1), (2, -1), (3, None), (4, 7), (5, None), (6, 7), (7, None), (8, 7), (9, 0),
                       (9, 1), (9, 6), (9, 4), (10, None)]),
    "cf_residual_tc": ((8, 6, 2, P, 8, P, 6, P, 8, P, 8, P, BIG, None),
                       [(1, -1), (2, -1), (3, -1), (4, None), (5, 7), (6, None), (7, 5), (8, None), (9, 7),
                        (10, None), (11, 7)]),
    "cf_trsv_f32": ((0, 8, 2, P, 8, P, 8, P, BIG, None),
                    [(1, -1), (1, 4), (2, -1), (3, -1), (3, 17), (4, None), (5, 7), (6, None), (7, 7)]),
    "cf_trsv_f32_withheld": ((0, 8, 2, P, 8, P, 8, 0, P, BIG, None),
                             [(1, -1), (1, 4), (2, -1), (3, 17), (4, None), (5, 7), (6, None), (7, 7), (8, -1)]),
    "cf_posv_mixed": ((8, 2, P, 8, P, 8, P, 8, 3, P, None, P, BIG, None, None),
                      [(1, -1), (2, -1), (3, None), (4, 7), (5, None), (6, 7), (7, None), (8, 7), (9, 0),
                       (9, 6), (10, None)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_invalid_argument_returns_its_position(name):
    base, bad = CASES[name]
    fn = getattr(L, name)
    assert len(base) == len(fn.argtypes)
    for pos, val in bad:
        args = list(base)
        args[pos - 1] = val
        assert fn(*args) == -pos, (name, pos, val)


def test_every_entry_point_with_arguments_is_covered():
    skip = {"cf_default_options", "cf_status_string", "cf_last_cuda_error", "cf_kernel_launches",
            "cf_device_status", "cf_batched_autotune"}
    taking_args = {n for n in cf.header_functions() if not n.endswith("_workspace_size")} - skip
    assert taking_args <= set(CASES)


def test_autotune_argument_checks():
    n = (ctypes.c_int * 4)(16, 32, 64, 128)
    o = cf.options()
    fn = L.cf_batched_autotune
    assert fn(0, n, None, 0, 0, P, BIG, ctypes.byref(o), None, None) == -1
    assert fn(4, None, None, 0, 0, P, BIG, ctypes.byref(o), None, None) == -2
    assert fn(4, n, None, 3, 0, P, BIG, ctypes.byref(o), None, None) == -4
    assert fn(4, n, None, 0, 0, P, BIG, None, None, None) == -8


def test_bad_options_are_unsupported_before_any_cuda_call():
    # (a zero in v, leaf_h, arity, tol, max_iter or gmres_restart selects its default)
    for kw in ({"v": -1}, {"v": 129}, {"leaf_h": -1}, {"leaf_h": 513}, {"arity": 1}, {"arity": 9},
               {"outer_V": 100}, {"outer_V": -128}, {"gmres_restart": 257}, {"batch_cps": 9}, {"batch_cps": -1},
               {"fp64_residual": 2}, {"fp64_residual": -1}):
        assert L.cf_getrf(8, P, 8, P, P, P, BIG, _opt(**kw), None) == cf.CF_ERR_UNSUPPORTED, kw
        assert L.cf_potrf(8, P, 8, P, P, BIG, _opt(**kw), None) == cf.CF_ERR_UNSUPPORTED, kw
        assert L.cf_gesv_mixed(8, 2, P, 8, P, 8, P, 8, 3, P, None, P, BIG, _opt(**kw), None) == \
            cf.CF_ERR_UNSUPPORTED, kw


def test_tournament_shapes_per_routine():
    # FP64 routines: leaves <= 128 rows, arity <= 8; the mixed LU: v = 128
    # with leaves <= 256 and arity 2, or v <= 64 with leaves <= 512 and
    # arity * v <= 512
    for kw in ({"leaf_h": 129}, {"leaf_h": 512, "arity": 8}):
        assert L.cf_getrf(8, P, 8, P, P, P, BIG, _opt(**kw), None) == cf.CF_ERR_UNSUPPORTED, kw
        assert L.cf_getrf_noalloc(8, P, 8, P, P, _opt(**kw), None) == cf.CF_ERR_UNSUPPORTED, kw
        assert L.cf_getrf_workspace_size(1000, _opt(**kw)) == 0, kw
    for kw in ({"v": 128, "leaf_h": 257}, {"v": 128, "arity": 3}, {"v": 80, "leaf_h": 300},
               {"v": 64, "arity": 8, "leaf_h": 513}, {"v": 16, "arity": 8, "outer_V": 24}):
        assert L.cf_gesv_mixed(8, 2, P, 8, P, 8, P, 8, 3, P, None, P, BIG, _opt(**kw), None) == \
            cf.CF_ERR_UNSUPPORTED, kw
        assert cf.gesv_mixed_workspace_size(1000, 1, "f16", **kw) == 0, kw
    assert cf.gesv_mixed_workspace_size(1000, 1, "f16", v=64, leaf_h=512, arity=8) > 0
    # left 0, the mixed LU takes v = 64, leaves of 512 rows, arity 8; v = 128 alone takes 256 / 2
    assert cf.gesv_mixed_workspace_size(1000, 1, "f16") == cf.gesv_mixed_workspace_size(1000, 1, "f16", v=64,
                                                                                         leaf_h=512, arity=8)
    assert cf.gesv_mixed_workspace_size(1000, 1, "f16", v=128) == cf.gesv_mixed_workspace_size(1000, 1, "f16", v=128,
                                                                                                leaf_h=256, arity=2)
    assert cf.gesv_mixed_workspace_size(1000, 1, "f16", v=32, leaf_h=512, arity=16) == 0
    assert cf.posv_mixed_workspace_size(1000, 1, "f16", leaf_h=512, arity=8) > 0   # no tournament


def test_fp64_leaves_at_most_128_rows():
    # the mixed solvers take leaves of up to 256 rows, the FP64 routines 128
    assert L.cf_getrf(8, P, 8, P, P, P, BIG, _opt(leaf_h=200), None) == cf.CF_ERR_UNSUPPORTED
    assert L.cf_getrf_noalloc(8, P, 8, P, P, _opt(leaf_h=129), None) == cf.CF_ERR_UNSUPPORTED
    assert L.cf_getrf_workspace_size(1000, _opt(leaf_h=129)) == 0
    assert L.cf_getrf_workspace_size(1000, _opt(leaf_h=128)) > 0
    assert cf.gesv_mixed_workspace_size(1000, 1, "f16", leaf_h=256) > 0


def test_zero_fields_select_defaults():
    z = cf.Options()                      # every field 0
    d = cf.options()
    assert L.cf_getrf_workspace_size(4096, ctypes.byref(z)) == L.cf_getrf_workspace_size(4096, ctypes.byref(d)) > 0


def test_fp8_updates_are_cholesky_only():
    assert L.cf_gesv_mixed(256, 2, P, 256, P, 256, P, 256, 4, P, None, P, BIG, None, None) == -9
