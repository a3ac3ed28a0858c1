"""The benchmark's nominal per-pass model and kind names (host only).

`bench.pass_flops_bytes` counts the algorithmic FLOPs and bytes a pass kind
must do (the roofline's numerator) and `bench.kind_name` names the kernel a
kind ran; both read the pass flags the library reports (1 inverse FFT first,
2 forward FFT, 4 kinetic phase and inverse FFT, 16 the phase of one axis,
256/512 one or two potential tables)."""
import math

import bench


def _kind(axis, flags, surfaces=3, variant=0):
    return {"axis": axis, "flags": flags, "surfaces": surfaces, "variant": variant}


def test_fft_only_pass_counts_one_fft_and_the_psi_round_trip():
    n, S = (64, 64, 64), 3
    f, b = bench.pass_flops_bytes(_kind(1, 2, surfaces=1), n, S, 16)
    amps = S * 64 ** 3
    assert f == amps // 64 * 5 * 64 * math.log2(64)
    assert b == 2 * 16 * amps


def test_potential_pass_counts_the_matvec_and_the_packed_table():
    n, S = (64, 64, 64), 3
    P = 64 ** 3
    f, b = bench.pass_flops_bytes(_kind(0, 1 | 2 | 256), n, S, 16)
    assert f == 2 * (S * P // 64) * 5 * 64 * 6 + (8 * S * S - 2 * S) * P
    assert b == 2 * 16 * S * P + 16 * (S * (S + 1) // 2) * P


def test_kinetic_table_bytes_joint_against_per_axis():
    n, S = (128, 128, 128), 3
    P = 128 ** 3
    _, joint = bench.pass_flops_bytes(_kind(2, 2 | 4, surfaces=1), n, S, 8)
    _, axes = bench.pass_flops_bytes(_kind(2, 2 | 4 | 16, surfaces=1), n, S, 8)
    assert joint - axes == 8 * P - 8 * 128   # a phase per grid point against one per line point


def test_kind_names(monkeypatch):
    monkeypatch.setattr(bench, "N_GRID", (64, 64, 64))
    monkeypatch.setitem(bench.W, "fp32", False)
    assert bench.kind_name(_kind(0, 1 | 2 | 256)) == "axis_pass_kernel<L=64,SV=3> [I0 V F0]"
    assert bench.kind_name(_kind(0, 1 | 2 | 256 | 512, variant=2)) == "axis_pass_tma_kernel<L=64,SV=3> [I0 VV F0]"
    assert bench.kind_name(_kind(2, 2 | 4, 1, 4)) == "axis_pass_reg_kernel<L=64,SV=1> [F2 T I2]"
    assert bench.kind_name(_kind(1, 2 | 4 | 16, 1, 4)) == "axis_pass_reg_kernel<L=64,SV=1> [F1 T1 I1]"
    assert bench.kind_name(_kind(0, 2 | 4 | 16 | 256, 3, 4)) == "axis_pass_reg_kernel<L=64,SV=3> [V F0 T0 I0]"


def test_plane_pass_counts_both_axes(monkeypatch):
    n, S = (128, 128, 128), 3
    amps = S * 128 ** 3
    f, b = bench.pass_flops_bytes(_kind(1, 2 | 4 | 16 | 32, surfaces=1, variant=0), n, S, 8)
    f1, b1 = bench.pass_flops_bytes(_kind(1, 2 | 4 | 16, surfaces=1), n, S, 8)
    f2, b2 = bench.pass_flops_bytes(_kind(2, 2 | 4 | 16, surfaces=1), n, S, 8)
    assert f == f1 + f2                     # the two line passes' arithmetic
    assert b == b1 + b2 - 2 * 8 * amps      # one psi round trip instead of two
    monkeypatch.setattr(bench, "N_GRID", n)
    monkeypatch.setitem(bench.W, "fp32", True)
    assert bench.kind_name(_kind(1, 2 | 4 | 16 | 32, 1, 0)) == \
        "axis_pass_plane_kernel<LA=128,LB=128,float2> [F1 T1 I1 F2 T2 I2]"


def test_joint_plane_pass_counts_three_line_passes(monkeypatch):
    n, S = (64, 64, 64), 3
    amps = S * 64 ** 3
    f, b = bench.pass_flops_bytes(_kind(1, 2 | 4 | 32, surfaces=1), n, S, 16)
    parts = [bench.pass_flops_bytes(_kind(1, 2, surfaces=1), n, S, 16),
             bench.pass_flops_bytes(_kind(2, 2 | 4, surfaces=1), n, S, 16),
             bench.pass_flops_bytes(_kind(1, 1, surfaces=1), n, S, 16)]
    assert f == sum(p[0] for p in parts)
    assert b == sum(p[1] for p in parts) - 4 * 16 * amps  # one psi round trip instead of three
    monkeypatch.setattr(bench, "N_GRID", n)
    monkeypatch.setitem(bench.W, "fp32", False)
    assert bench.kind_name(_kind(1, 2 | 4 | 32, 1, 0)) == "axis_pass_plane_joint_kernel<LA=64,LB=64> [F1 F2 T I2 I1]"
