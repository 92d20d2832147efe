"""Helpers for the GPU parity tests: upload seeded inputs, run the CUDA path
through the C ABI, compare with the oracle."""
import numpy as np
import torch

PLANES = ["r", "g", "b", "alpha", "depth", "invdepth", "median", "nx", "ny", "nz", "distortion",
          "T_final"]
DEPTH_PLANES = (4, 5, 6, 10)  # planes that switch value with the object/screen branch
TOL_ABS = 2e-5  # channel tolerance; planes whose values exceed 1 scale it by |value|


def to_dev(scene, device="cuda"):
    keys = ("mu", "quat", "scale", "opacity", "sh")
    return {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(device) for k in keys}


def gpu_scene(scene, settings=None, device="cuda"):
    from paper_2411_00771_gb300 import binding as B
    d = to_dev(scene, device)
    s = B.default_settings(**(settings or {}))
    sc = B.Scene(d["mu"], d["quat"], d["scale"], d["opacity"], d["sh"], scene["sh_degree"], s)
    return sc, d


def gpu_render(scene, cam, settings=None):
    from paper_2411_00771_gb300 import binding as B
    sc, d = gpu_scene(scene, settings)
    H, W = cam["height"], cam["width"]
    cnt = torch.empty((H, W), dtype=torch.int32, device="cuda")
    out, frame = sc.render(cam, n_contrib=cnt)
    torch.cuda.synchronize()
    return sc, d, out, cnt, frame


def channel_errors(gpu_out, ref_out, mask=None):
    """Per-plane max |gpu - ref| / max(1, |ref|) over pixels in mask."""
    g = np.asarray(gpu_out, np.float64)
    r = np.asarray(ref_out, np.float64)
    e = np.abs(g - r) / np.maximum(1.0, np.abs(r))
    if mask is not None:
        e = e[:, mask]
    return e.reshape(e.shape[0], -1).max(axis=1) if e.size else np.zeros(g.shape[0])


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
