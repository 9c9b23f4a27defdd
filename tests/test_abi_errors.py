"""Error behaviour of the C ABI that needs no GPU: invalid arguments return
FS_EINVAL with a message naming the entry point (fs_last_error), before any
device call; NULL handles are no-ops for the destroy calls; the pure helpers
answer from their arguments alone."""
import ctypes as C

import pytest

from paper_2407_10797_gb300 import fstat

EINVAL = -1


@pytest.fixture(scope="module")
def L():
    return fstat.load()


def err(L):
    return L.fs_last_error().decode()


def test_plan_create_rejects_bad_grids_and_modes(L):
    h = C.c_void_p()
    cases = [
        (0, 0.01, 1e-6, 1e7, 0, "n_bins > 0"),
        (100, 0.0, 1e-6, 1e7, 0, "f_min"),
        (100, 0.01, -1e-6, 1e7, 0, "df"),
        (100, 0.01, 1e-6, float("nan"), 0, "T_obs"),
        (100, 0.01, 1e-6, 1e7, 7, "unknown mode"),
        (1 << 31, 0.01, 1e-6, 1e7, 1, "2^31"),
        ((1 << 40) + 1, 0.01, 1e-6, 1e7, 0, "too large"),
    ]
    for n, fmin, df, T, mode, word in cases:
        assert L.fs_plan_create(C.byref(h), n, fmin, df, T, mode, None) == EINVAL
        assert h.value is None
        assert "fs_plan_create" in err(L) and word in err(L), (n, err(L))
    assert L.fs_plan_create(None, 100, 0.01, 1e-6, 1e7, 0, None) == EINVAL


def test_calls_on_a_null_plan_are_refused(L):
    assert L.fs_fstat_batch(None, None, 4, None, 1, None, None) == EINVAL
    assert L.fs_amplitudes(None, None, 4, None, 1, None, None, None) == EINVAL
    assert "fs_amplitudes" in err(L)
    assert L.fs_graph_run(None, 1) == EINVAL
    assert L.fs_plan_destroy(None) == 0
    assert L.fs_mlp_destroy(None) == 0


def test_response_model_arguments_are_checked(L):
    for N, K, word in ((3, 0, "filter order"), (-2, 0, "filter order"), (1, 2, "k_max"), (0, -1, "k_max"),
                       (2, 1, "plan is NULL")):
        assert L.fs_plan_set_response(None, N, K) == EINVAL
        assert "fs_plan_set_response" in err(L) and word in err(L), (N, K, err(L))
    n, k = C.c_int(), C.c_int()
    assert L.fs_plan_get_response(None, C.byref(n), C.byref(k)) == EINVAL


def test_orbit_arguments_are_checked(L):
    for e, word in ((-1e-3, "eccentricity"), (0.06, "eccentricity"), (float("nan"), "eccentricity"),
                    (0.0048, "plan is NULL")):
        assert L.fs_plan_set_orbit(None, C.c_double(e)) == EINVAL
        assert "fs_plan_set_orbit" in err(L) and word in err(L), (e, err(L))
    v = C.c_double()
    assert L.fs_plan_get_orbit(None, C.byref(v)) == EINVAL
    assert L.fs_plan_selftest_timeout(None) == EINVAL and "fs_plan_selftest_timeout" in err(L)
    for a, word in ((-1.0, "arm length"), (101.0, "arm length"), (float("inf"), "arm length"),
                    (8.339, "plan is NULL")):
        assert L.fs_plan_set_arm(None, C.c_double(a)) == EINVAL
        assert "fs_plan_set_arm" in err(L) and word in err(L), (a, err(L))
    assert L.fs_plan_get_arm(None, C.byref(v)) == EINVAL


def test_network_creation_rejects_bad_shapes(L):
    h = C.c_void_p()
    for width, batch in ((7, 16), (2048, 16), (0, 16), (64, 0)):
        assert L.fs_mlp_create(C.byref(h), width, batch, 1, None) == EINVAL
        assert h.value is None and "fs_mlp_create" in err(L)
    for groups in (0, 1025):
        assert L.fs_mlp_create_group(C.byref(h), groups, 64, 16, 1, None) == EINVAL
        assert h.value is None and "fs_mlp_create_group" in err(L)


def test_pure_helpers(L):
    assert L.fs_mlp_num_params(0) == -1
    W = 256
    assert L.fs_mlp_num_params(W) == W * 5 + W + 2 * (W * W + W) + W + 1
    assert L.fs_mlp_groups(None) == -1


def test_noalloc_limits_are_checked_first(L):
    F = C.c_void_p(8)   # never dereferenced: the size checks come first
    assert L.fs_fstat_batch_noalloc(32769, 0.01, 1e-6, 1e7, F, F, F, 4, None, 8, F, None, None) == EINVAL
    assert "limit" in err(L)
    assert L.fs_fstat_batch_noalloc(1000, 0.01, 1e-6, 1e7, F, F, F, 1025, None, 8, F, None, None) == EINVAL
    assert L.fs_fstat_batch_noalloc(1000, 0.01, 1e-6, 1e7, F, F, F, 4, None, 65, F, None, None) == EINVAL
    assert L.fs_fstat_batch_noalloc(1000, 0.01, 1e-6, 1e7, None, F, F, 4, None, 8, F, None, None) == EINVAL
    assert L.fs_fstat_batch_noalloc(1000, 0.01, 1e-6, 1e7, F, F, F, 0, None, 8, F, None, None) == 0   # B = 0


def test_channel_sets_probe_and_check_refuse_bad_arguments(L):
    h = C.c_void_p()
    assert L.fs_plan_create_tdi(C.byref(h), 100, 0.01, 1e-6, 1e7, 0, 7, None) == EINVAL
    assert h.value is None and "fs_plan_create_tdi" in err(L) and "channel set" in err(L)
    assert L.fs_plan_create_tdi(C.byref(h), 0, 0.01, 1e-6, 1e7, 0, 1, None) == EINVAL   # the grid checks apply too
    assert L.fs_plan_channels(None) == -1
    assert L.fs_plan_check(None, None) == EINVAL and "fs_plan_check" in err(L)
    assert L.fs_mixed_probe(None, None, 1, None, 1, 0, 0, 10, None) == EINVAL and "fs_mixed_probe" in err(L)
    assert L.fs_plan_set_data(None, None, None, None) == EINVAL and "fs_plan_set_data" in err(L)


def test_swarm_dimensions_are_checked(L):
    """A swarm declares 5 or 6 dimensions (0 reads as 5); anything else is
    refused before any launch (the plan is checked first, so a fake non-NULL
    plan handle is never dereferenced on this path)."""
    buf = (C.c_double * 64)()
    p = C.cast(buf, C.c_void_p).value
    for dims, ok in ((7, False), (4, False), (-1, False)):
        sw = fstat.fs_swarm(1, 1, p, p, p, p, p, p, 1.0, None, 0, dims)
        assert L.fs_pso_best(C.c_void_p(8), C.byref(sw), C.c_void_p(p), C.c_void_p(p)) == EINVAL
        assert "dims" in err(L)
