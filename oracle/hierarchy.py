"""Chunk / keyframe pose composition (oracle).

Sec. 4.2: a chunk's local solve is relative to its first frame (identity initial
poses); the chunk's keyframe is that first frame.  A new global keyframe is
initialised with the intra-chunk delta of the preceding chunk composed with the
previous global keyframe pose, and after the global solve every frame's world pose
is its keyframe's global pose composed with its local pose:
    T_world(f) = T_kf(global) T_local(f).
"""
import numpy as np


def keyframe_init(prev_kf_world, local_delta):
    """Initial world pose of the next keyframe: previous keyframe pose composed with the chunk delta."""
    return np.asarray(prev_kf_world) @ np.asarray(local_delta)


def compose(kf_world, local):
    """World pose of a chunk member from its keyframe's world pose and its local pose."""
    return np.asarray(kf_world) @ np.asarray(local)
