"""CPU tests of the benchmark's roofline arithmetic: the support-node count
against a direct enumeration, and the byte models of the stream-collide and
the cell kernels against hand counts."""
import numpy as np

import bench


def test_support_nodes_counts_distinct_nodes():
    # one point: W^3 nodes; two points one spacing apart in x share W^2 (W - 1)
    y = np.array([[5.5, 6.25, 7.75]])
    assert bench.support_nodes(y, (16, 16, 16), 2) == 8
    assert bench.support_nodes(y, (16, 16, 16), 4) == 64
    y2 = np.vstack([y, y + [1.0, 0.0, 0.0]])
    assert bench.support_nodes(y2, (16, 16, 16), 2) == 8 + 4
    assert bench.support_nodes(y2, (16, 16, 16), 4) == 64 + 16
    # periodic wrap in x and z: a point at the upper seam
    ys = np.array([[15.5, 3.0, 15.2]])
    assert bench.support_nodes(ys, (16, 16, 16), 2) == 8


def test_support_nodes_against_enumeration():
    rng = np.random.default_rng(3)
    dims = (12, 10, 9)
    y = rng.uniform([0, 2, 0], [12, 7, 9], size=(40, 3))
    for w in (2, 4):
        nodes = set()
        for p in y:
            b = np.floor(p).astype(int) - (w // 2 - 1)
            for dz in range(w):
                for dy in range(w):
                    for dx in range(w):
                        nodes.add(((b[0] + dx) % dims[0], b[1] + dy, (b[2] + dz) % dims[2]))
        assert bench.support_nodes(y, dims, w) == len(nodes)


def test_byte_models():
    # 19 FP32 populations read and written
    assert bench.POP_BYTES_PER_NODE == 2 * 19 * 4
    # near field: + float4 force read + float4 velocity store
    assert bench.NEAR_BYTES_PER_NODE == 152 + 16 + 16
    # per tet: int4 indices, 3 float4 B rows, 4 float4 corner forces written and read, 4 int32 entries
    assert bench.CELL_BYTES_PER_TET == 16 + 3 * 16 + 2 * 4 * 16 + 4 * 4
    # per vertex: xr + u (K1), row bounds, xr + u (K23), vertex force; plus one float4 per support node
    assert bench.cell_bytes(0, 1, 2) == 32 + 8 + 32 + 16 + 8 * 16
    assert bench.cell_bytes(10, 3, 4) == 10 * 208 + 3 * (88 + 64 * 16)


def test_host_replicas_are_capped_by_cores_and_memory():
    import os

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    assert 1 <= bench._host_replicas(32**3) <= cores
    # a lattice whose oracle would not fit twice into any host's memory: one replica
    assert bench._host_replicas(10**13) == 1


def test_region_statistics_take_the_median_of_the_regions():
    st = bench.region_stats([3.0, 1.0, 2.0, 10.0, 2.5], 20)
    assert st["n"] == 5 and st["steps_per_region"] == 20
    assert st["ms_per_step_median"] == 2.5 / 20
    assert st["ms_per_step_min"] == 1.0 / 20 and st["ms_per_step_max"] == 10.0 / 20


class _WL:
    nx, ny, nz, delta = 16, 16, 16, 2
    n_nodes = 16 ** 3


def test_stream_collide_roofline_picks_the_longer_part_and_counts_its_bytes():
    y = np.array([[5.5, 6.25, 7.75], [9.2, 8.1, 3.3]])
    n_sup = bench.support_nodes(y, (16, 16, 16), 2)
    # far field longer: 152 B per node outside the region (FP32), 76 with 16-bit storage
    r = bench.stream_collide_roofline(_WL, [0, 0, 0.05, 0.01, 0], 1000, y, "f32", 6000.0)
    assert r["kernel"] == "k_lbm_far" and r["units_per_launch"] == 16 ** 3 - 1000
    assert r["algorithmic_bytes_per_launch"] == 152 * (16 ** 3 - 1000)
    assert abs(r["achieved"] - 152 * (16 ** 3 - 1000) / 0.05e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    r16 = bench.stream_collide_roofline(_WL, [0, 0, 0.05, 0.01, 0], 1000, y, "f16sr", 6000.0)
    assert r16["bytes_per_unit"] == 76
    # near field longer: 184 B per region node (+16 B per support node whose force is zeroed)
    r = bench.stream_collide_roofline(_WL, [0, 0, 0.01, 0.05, 0], 1000, y, "f32", 6000.0)
    assert r["kernel"] == "k_lbm_near" and r["units_per_launch"] == 1000
    assert r["algorithmic_bytes_per_launch"] == 184 * 1000 + 16 * n_sup
    r16 = bench.stream_collide_roofline(_WL, [0, 0, 0.01, 0.05, 0], 1000, y, "bf16", 6000.0)
    assert r16["bytes_per_unit"] == 76 + 32


def test_sweep_cases_cover_the_capillary_numbers_and_weights():
    assert bench.SWEEP_CA == (0.05, 0.2, 0.5) and bench.SWEEP_W == (0.0, 0.5, 1.0)
    # the paper's own shear runs: neo-Hookean (w = 1) over a range of Ca
    assert bench.PAPER_SWEEP_CA == (0.05, 0.1, 0.2, 0.3, 0.5)


def test_step_roofline_adds_every_kernel_of_the_step():
    class WL(_WL):
        n_tets, n_verts = 100, 30

    roof = {"near_region_nodes": 1000, "support_nodes": 50}
    r = bench.step_roofline(WL, roof, "f32", 0.02, 6000.0)
    far = 152 * (16 ** 3 - 1000)
    near = 184 * 1000 + 16 * 50
    cells = 100 * 208 + 30 * (88 + 8 * 16)
    interp = 30 * (48 + 8 * 16)
    assert r["parts"] == {"far": far, "near": near, "cells": cells, "interp": interp}
    assert r["algorithmic_bytes_per_step"] == far + near + cells + interp
    assert abs(r["frac"] - (far + near + cells + interp) / 0.02e-3 / 1e9 / 6000.0) < 1e-12
    # 16-bit storage halves the population bytes only
    r16 = bench.step_roofline(WL, roof, "f16sr", 0.02, 6000.0)
    assert r16["parts"]["far"] == far // 2 and r16["parts"]["near"] == near - 76 * 1000
