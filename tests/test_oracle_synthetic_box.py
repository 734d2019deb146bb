"""The exact room-box depth used to test tracking: every back-projected pixel lies
on a face of the box, and the nearest face along its ray."""
import numpy as np

from paper_2503_01109_gb300 import synthetic as syn


def test_box_depth_points_lie_on_the_first_face():
    for cam in syn.corner_trajectory(3, 64, 48, 52.5) + [syn.room_camera(64, 48, 52.5, seed=4)]:
        d = syn.box_depth(cam).astype(np.float64)
        M = np.asarray(cam["world_to_cam"], np.float64).reshape(3, 4)
        R, t = M[:, :3], M[:, 3]
        ys, xs = np.mgrid[0:48, 0:64]
        pc = np.stack([(xs - cam["cx"]) / cam["fx"] * d, (ys - cam["cy"]) / cam["fy"] * d, d], -1)
        pw = (pc - t) @ R
        gap = np.abs(np.abs(pw) - syn.ROOM_HALF).min(-1)      # distance to the nearest face plane
        assert gap.max() < 1e-5
        assert np.all(np.abs(pw) <= syn.ROOM_HALF + 1e-5)      # inside the box: the first face hit
