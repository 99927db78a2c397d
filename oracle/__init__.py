"""FP64 CPU oracle of the batched Gaussian-splatting renderer -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this package.
The product path (the CUDA library and its Python binding) never imports, links or calls it,
and this package imports nothing from the product: scenes are read by duck typing from any
object with the attributes of a `Scene` (nodes with SoA arrays, env_node_ids, node_poses,
cams_per_env, cam_intr, cam_res, cam_pose).

The rendering arithmetic lives in oracle.cpp (plain FP64 C++, std::thread over pixel rows);
see its header for the definition it implements and the readings it fixes.  The image
randomisation applied to rendered frames is augment.py (numpy, FP64); LiDAR ray tracing of the
same Gaussians is lidar.cpp / lidar.py (FP64 C++, brute force over the env's Gaussians); the
mesh -> Gaussian transfer is mesh.py and depth -> TSDF fusion tsdf.py (numpy, FP64).
"""
from . import augment, lidar, mesh, tsdf
from .oracle import (OracleOptions, build, lib_path, project_view, render_view, backward_view,
                     backward_scene, pose_twist_grad, sh_basis)

__all__ = ["OracleOptions", "augment", "lidar", "mesh", "tsdf", "build", "lib_path", "project_view", "render_view", "backward_view",
           "backward_scene", "pose_twist_grad", "sh_basis"]
