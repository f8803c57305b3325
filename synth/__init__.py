"""Seeded synthetic inputs for the elevation-mapping fusion path.

This module holds none of the fusion method's arithmetic.  It simulates
terrain and range sensors and hands out sensor-frame point clouds with their
sensor-to-map poses.  The tests, the smoke check and the benchmark draw their
inputs from here, so the oracle and the CUDA path see the same data.

The recorded robot logs the paper measures on (ANYmal with Bpearl LiDARs or
four Realsense cameras, Section III) are not available; these generators stand
in for them with the same shapes: depth images with invalid pixels, spinning
LiDAR scans, terrain with steps, boxes, stairs and ramps.
"""
from .terrain import (Terrain, StairsTerrain, raycast, pose_matrix, single_update, DepthRig, depth_stream,
                      LidarRig, lidar_stream, scattered_cloud, batch_clouds, random_prior)

__all__ = ["Terrain", "StairsTerrain", "raycast", "pose_matrix", "single_update", "DepthRig", "depth_stream",
           "LidarRig", "lidar_stream", "scattered_cloud", "batch_clouds", "random_prior"]
