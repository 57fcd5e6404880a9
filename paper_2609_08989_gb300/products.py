"""Image products of a traced camera (paper Sec. 4.2): per-pixel maps as 2-D
arrays, the Doppler on/off pair of one scene, and an .npz file holding the
maps with the scene's parameters.

A traced camera's outputs are flat, pixel p = j * nx + i with j ascending in
beta; ``image`` reshapes one field to [ny, nx] (row j = beta_j, column i =
alpha_i).  Plotting (colour maps, contours) is left to the caller.
"""
from __future__ import annotations

import dataclasses
import json
from typing import Dict, Optional

import numpy as np

from . import scenes
from . import tartarus as T

MAPS = ("intensity", "code", "n_cross", "h_max", "steps")


def image(out: Dict, sc: scenes.Scene, field: str = "intensity", k: Optional[int] = None) -> np.ndarray:
    """One output field as an [ny, nx] numpy array; k selects a crossing slot of
    r_cross / g / I_cross."""
    v = out[field]
    v = v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)
    if v.ndim == 2:
        if k is None:
            raise ValueError("crossing fields need a slot k")
        v = v[k]
    if v.size != sc.nx * sc.ny:
        raise ValueError("outputs hold %d pixels, the camera %d" % (v.size, sc.nx * sc.ny))
    return v.reshape(sc.ny, sc.nx)


def render(sc: scenes.Scene, stream=None, tune=None) -> Dict[str, np.ndarray]:
    """Trace the scene on the current GPU and return its maps as [ny, nx] arrays
    (the per-pixel fields plus r_cross / g / I_cross of the first crossing)."""
    import torch
    out = T.trace(sc, stream=stream, tune=tune)
    torch.cuda.synchronize()
    maps = {f: image(out, sc, f) for f in MAPS}
    for f in ("r_cross", "g", "I_cross"):
        maps[f + "0"] = image(out, sc, f, 0)
    return maps


def doppler_pair(sc: scenes.Scene, **kw) -> Dict[str, Dict[str, np.ndarray]]:
    """The scene with and without the Doppler factor (paper Fig. 3a and 3b)."""
    return {"doppler": render(sc.replace(doppler=1), **kw), "no_doppler": render(sc.replace(doppler=0), **kw)}


def left_right_ratio(intensity: np.ndarray, sc: scenes.Scene) -> float:
    """Summed intensity of the alpha < 0 half over the alpha > 0 half."""
    alpha = sc.alpha_min + (np.arange(sc.nx) + 0.5) * (sc.alpha_max - sc.alpha_min) / sc.nx
    return float(intensity[:, alpha < 0].sum() / intensity[:, alpha > 0].sum())


def save_npz(path: str, sc: scenes.Scene, maps: Dict[str, np.ndarray]) -> None:
    """Write the maps and the scene parameters (JSON, without a metric table)."""
    meta = {k: v for k, v in dataclasses.asdict(sc).items() if k != "table"}
    np.savez_compressed(path, scene=json.dumps(meta), **maps)


def main(argv=None) -> int:
    import argparse
    p = argparse.ArgumentParser(description="Render a paper scene to an .npz of per-pixel maps.")
    p.add_argument("scene", choices=["e3", "e3_nodoppler", "e5", "osiris", "kerr_disk"])
    p.add_argument("--n", type=int, default=1024)
    p.add_argument("--out", required=True)
    a = p.parse_args(argv)
    make = {"e3": lambda n: scenes.kerr_e3(n), "e3_nodoppler": lambda n: scenes.kerr_e3(n, doppler=0),
            "e5": scenes.schwarzschild_e5, "osiris": scenes.osiris_scene, "kerr_disk": scenes.kerr_disk}
    sc = make[a.scene](a.n)
    save_npz(a.out, sc, render(sc))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
