"""Seeded synthetic inputs (scenes, trajectories, depth images) shared by
the CPU oracle's tests and the CUDA path.  Holds none of the method's
arithmetic."""
from .scenes import Camera, Frame, GridSpec, Workload, body_pose, make  # noqa: F401
