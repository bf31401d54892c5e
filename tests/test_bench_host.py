"""Host logic of bench.py that turns ncu output into the committed figures:
the kernel-name parsing that maps a captured launch to its sweep direction
and precision, and the per-kernel summary of a launch list."""
import pytest

bench = pytest.importorskip("bench")


@pytest.mark.parametrize("name,kind", [
    ("void sldg::k_sweep_x12_df<3, 2, 0, 1, 1>(const double *, double *, int, int, int, int)", ("x12", "fp64")),
    # a parameter list naming double does not make an FP32 kernel FP64
    ("void sldg::k_sweep_x12_f32<3, 2, 0, 0>(const float *, float *, int, const double *, const double *)",
     ("x12", "fp32")),
    ("void sldg::k_rho_partial<float, 0>(const T1 *, long long, long long, long long, const float2 *, double *)",
     ("rho", "fp32")),
    ("void sldg::k_rho_partial<double, 1>(const T1 *, long long, long long, long long, const float2 *, double *)",
     ("rho", "fp64")),
    ("void sldg::k_sweep_strided_df3<3, 0, 1, 1, 1>(const double *, double *, int, long long)", ("v", "fp64")),
    ("void sldg::k_sweep_strided_df3<3, 1, 0, 1, 1>(const double *, double *, int, long long)", ("x2", "fp64")),
    ("void sldg::k_sweep_strided_f2<2, 0, 1>(const float *, float *, int, long long)", ("v", "fp32")),
    ("void sldg::k_sweep_x1_warp<4, 1, 1, 1>(double *, int, long long, int)", ("x1", "fp64")),
    ("void sldg::k_sweep_x1_f2warp<2>(float *, int, long long)", ("x1", "fp32")),
    ("void sldg::<unnamed>::k_spline_sweep<float, 1, 0, 1, 0>(float *, int, long long)", ("x1", "fp32")),
    ("void sldg::<unnamed>::k_spline_sweep<float, 0, 0, 1, 0>(float *, int, long long)", ("x2", "fp32")),
    ("void sldg::<unnamed>::k_spline_sweep<double, 0, 1, 1, 1>(double *, int, long long)", ("v", "fp64")),
    ("void sldg::k_pois_fwd_x(const double *, double *)", None),
])
def test_kernel_kind(name, kind):
    assert bench._kernel_kind(name) == kind


def test_summarize_launches(tmp_path, capsys):
    # ncu --csv launch list: one row per launch, times in the unit ncu chose
    rows = [
        '"ID","Process ID","Kernel Name","Metric Name","Metric Unit","Metric Value"',
        '"0","1","void sldg::k_sweep_x12_df<3, 2, 0, 1, 1>(const double *)","gpu__time_duration.sum","ms","30.5"',
        '"1","1","void sldg::k_rho_partial<double, 1>(const double *)","gpu__time_duration.sum","us","6,100"',
        '"2","1","void sldg::k_sweep_x12_df<3, 2, 0, 1, 1>(const double *)","gpu__time_duration.sum","ns","29500000"',
        '"3","1","void sldg::k_energy(const double *)","gpu__time_duration.sum","nsecond","1000"',
    ]
    p = tmp_path / "launches.csv"
    p.write_text("\n".join(rows) + "\n")
    bench.summarize_launches(str(p))
    out = capsys.readouterr().out
    assert out.startswith("4 launches, 66.10 ms of device time")
    lines = [l for l in out.splitlines() if l.startswith("| `")]
    assert lines[0] == "| `k_sweep_x12_df<3, 2, 0, 1, 1>` | 2 | 60.000 | 90.8% |"
    assert lines[1] == "| `k_rho_partial<double, 1>` | 1 | 6.100 | 9.2% |"
    assert lines[2].startswith("| `k_energy` | 1 | 0.001 |")
