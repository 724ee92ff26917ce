"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds scene geometry only: cameras, analytic depth maps (ray casting of
a sphere or of a height-field terrain with box buildings), brick lists, and
synthetic histogram counts for chunk workloads.  It contains none of the
method's arithmetic (no binning, no TGV operator, no prox): both the oracle and
the CUDA library consume what it produces and compute everything else on their
own.

The scenes stand in for the paper's datasets (close-range Citywall/Breisach and
aerial Copenhagen, Sec. 5 and the supplementary), which are not available here.
"""
from .scenes import (  # noqa: F401
    Camera,
    DomainDesc,
    Scene,
    dense_bricks,
    look_at,
    pinhole_intrinsics,
    sphere_scene,
    lidar_sphere_scene,
    spherical_scanner,
    terrain_scene,
    terrain_lidar_scans,
    plane_depth,
    random_histograms,
    chunk_workload,
    chunk_histogram,
    synthetic_votes_torch,
    multilevel_scene,
    ChunkSpec,
    CONFIG_SEEDS,
)
