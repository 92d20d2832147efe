"""Hand-built scenes for the oracle pins (closed-form cases)."""
import math

import numpy as np

SQRT_PI2 = 2.0 * math.sqrt(math.pi)


def make_scene(surfels, sh_degree=0):
    """surfels: list of dict(mu, quat=(w,x,y,z), scale=(su,sv), opacity, rgb or sh)."""
    n = len(surfels)
    K = (sh_degree + 1) ** 2
    mu = np.zeros((n, 3)); q = np.zeros((n, 4)); s = np.zeros((n, 2)); o = np.zeros(n)
    sh = np.zeros((n, K, 3))
    for i, d in enumerate(surfels):
        mu[i] = d["mu"]
        q[i] = d.get("quat", (1.0, 0.0, 0.0, 0.0))
        s[i] = d["scale"]
        o[i] = d["opacity"]
        if "sh" in d:
            sh[i] = np.asarray(d["sh"]).reshape(K, 3)
        else:
            sh[i, 0] = (np.asarray(d.get("rgb", (0.5, 0.5, 0.5))) - 0.5) * SQRT_PI2
    return dict(mu=mu, quat=q, scale=s, opacity=o, sh=sh, sh_degree=sh_degree)


def camera(W=64, H=64, f=64.0, cx=None, cy=None):
    return dict(R=np.eye(3), t=np.zeros(3), fx=f, fy=f, cx=W / 2 if cx is None else cx,
                cy=H / 2 if cy is None else cy, width=W, height=H)


def pixel_grid(cam):
    W, H = cam["width"], cam["height"]
    x, y = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    return x, y
