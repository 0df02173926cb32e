"""Host-side helpers of bench.py (no GPU): the oracle baseline's scaling and
the preconditioner entry of the config."""
import argparse

import pytest


def test_growth_exponent_and_extrapolation():
    import bench
    assert bench.growth_exponent((1.0, 100), (8.0, 200)) == pytest.approx(3.0)
    n4 = 30000
    cb = bench.cpu_baseline_obj(2.0, n4, small=(0.25, n4 // 2))
    assert cb["growth_exponent"] == pytest.approx(3.0)
    # value is what was measured: the slice's own rate
    assert cb["value"] == pytest.approx(0.5) and cb["measured_on"] == "slice" and cb["slice_dofs"] == n4
    assert cb["value_linear_upper_bound"] == pytest.approx(1.0 / (2.0 * bench.PIPE["n_x"] / bench.SAMPLE_LAYERS))
    assert cb["value_extrapolated"] == pytest.approx(1.0 / (2.0 * (bench.FULL_DOFS / n4) ** 3.0))
    # an exponent above 1 makes the extrapolated rate the lower of the two full-size figures
    assert cb["value_extrapolated"] < cb["value_linear_upper_bound"] < cb["value"]
    assert "extrapolated" in cb["sample"] and "upper bound" in cb["sample"]
    assert cb["cores"] == 1 and cb["kind"] == "oracle"
    plain = bench.cpu_baseline_obj(2.0, n4)
    assert "value_extrapolated" not in plain


def test_pc_config_and_opts():
    import bench
    a = argparse.Namespace(precond=None, schur_agg=0)
    assert bench.pc_config(a)["precond"].startswith("auto") and bench.pc_opts(a) == {}
    a = argparse.Namespace(precond=4, schur_agg=0)
    assert bench.pc_config(a) == {"precond": "triangular-pmg + coarse Schur correction", "schur_agg": 16,
                                  "pressure_laplacian": "two-level: aggregates of 32 vertices, 8 + 8 smoothing steps"}
    assert bench.pc_opts(a) == {"precond": 4}
    a = argparse.Namespace(precond=4, schur_agg=64)
    assert bench.pc_opts(a) == {"precond": 4, "schur_agg": 64} and bench.pc_config(a)["schur_agg"] == 64
    a = argparse.Namespace(precond=None, schur_agg=0, lap_size=-1, lap_smooth=0, cheb_l=60)
    assert bench.pc_opts(a) == {"lap_size": -1, "cheb_l": 60}
    assert bench.pc_config(a)["pressure_laplacian"] == "chebyshev degree 60"
    a = argparse.Namespace(precond=1, schur_agg=0, lap_size=32, lap_smooth=4)
    assert bench.pc_opts(a) == {"precond": 1, "lap_size": 32, "lap_smooth": 4}
    assert "pressure_laplacian" not in bench.pc_config(a)
