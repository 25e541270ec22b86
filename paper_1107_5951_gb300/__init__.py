"""GB300-native voxel-gravity forward model (May & Knepley, arXiv 1107.5951).

The compute path is the CUDA library ``libgf.so`` (C ABI in ``include/gf.h``);
this package is its Python binding (:mod:`.gf`) plus the seeded synthetic
workload generators (:mod:`.workloads`).
"""
from .gf import (GfError, Plan, PointsPlan, hex_sources, gf_hex_sources, gf_plan_create_points, gf_adjoint, gf_forward, gf_last_error, gf_plan_bytes,  # noqa: F401
                 gf_plan_check, gf_plan_create, gf_plan_destroy, gf_plan_export_tree,
                 gf_plan_get_info, gf_plan_set_source_part, gf_plan_set_timing, gf_plan_stage_times, gf_version,
                 gf_launch_count, load, plan_bytes, Server, gf_server_create,
                 gf_server_submit, gf_server_wait, gf_server_stats_get, gf_server_destroy)

__all__ = ["GfError", "Plan", "PointsPlan", "hex_sources", "gf_hex_sources", "gf_plan_create_points", "gf_adjoint", "gf_forward", "gf_last_error", "gf_plan_bytes",
           "gf_plan_check", "gf_plan_create", "gf_plan_destroy", "gf_plan_export_tree",
           "gf_plan_get_info", "gf_plan_set_source_part", "gf_plan_set_timing", "gf_plan_stage_times", "gf_version",
           "gf_launch_count", "load", "plan_bytes", "Server", "gf_server_create",
           "gf_server_submit", "gf_server_wait", "gf_server_stats_get", "gf_server_destroy"]
