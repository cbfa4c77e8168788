"""Readers (and writers) of the input files of OpenCFD-FWH (Sec. III A, App. A).

* control.fwh (App. A1): a Fortran namelist with the run parameters
  (Kstep_start, Kstep_end, delta_step, FWH_data_Format, Mach number, AoA,
  time step, observer and frame counts, threads).  `read_control` returns
  every `key = value` pair of the namelist group(s), keys lower-cased.
* FWH_Surface_Geo.dat (App. A2, ASCII): a text line
  `variables=x,y,z,n1,n2,n3,dS`, then the number of Faces, then for each Face
  a line `nx ny nz` (one of them 1: a Face is a block face of the mesh)
  followed by its nx ny nz subfaces, one line of x y z n1 n2 n3 dS each.
* observers.dat (Sec. III A): one observer per row, x y z.
* FWH-xxxxxxxx.dat (App. A3; its figure is missing, so the layout below is a
  reading): one file per sampling frame, xxxxxxxx the iteration step (eight
  digits), holding the pulsations rho', u', v', w', p' of every subface in
  the order of FWH_Surface_Geo.dat.  FWH_data_Format 1 (ASCII): one subface
  per line, five numbers; lines that do not parse as numbers (headers) are
  skipped.  FWH_data_Format 0 (binary): the P x 5 values as little-endian
  FP64, subface-major, either raw or as one Fortran unformatted record (a
  4-byte length before and after).
* `load_dataset` stacks the frames Kstep_start, Kstep_start + delta_step, ...,
  Kstep_end into the library's field layout [nt][5][P] (float32 or float64),
  optionally into pinned host memory, reading the next frame on a thread
  while the current one is converted.

Nothing here computes any part of the FW-H path.
"""
from __future__ import annotations

import os
import re
import struct
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

GEO_HEADER = "variables=x,y,z,n1,n2,n3,dS"


@dataclass
class SurfaceGeo:
    centroids: np.ndarray   # [P][3]
    normals: np.ndarray     # [P][3]
    areas: np.ndarray       # [P]
    faces: list             # [(nx, ny, nz)] per Face, in file order

    @property
    def face_sizes(self) -> list:
        return [nx * ny * nz for nx, ny, nz in self.faces]

    @property
    def face_ranges(self) -> list:
        """Contiguous panel ranges [lo, hi) of the Faces."""
        out, lo = [], 0
        for n in self.face_sizes:
            out.append((lo, lo + n))
            lo += n
        return out


# ---------------------------------------------------------------- control ---

_NAMELIST_ITEM = re.compile(r"([A-Za-z_][A-Za-z0-9_%]*)\s*=\s*([^,\n/]+)")


def _nl_value(v: str):
    v = v.strip()
    low = v.lower()
    if low in (".true.", "t", ".t."):
        return True
    if low in (".false.", "f", ".f."):
        return False
    if len(v) >= 2 and v[0] == v[-1] and v[0] in "'\"":
        return v[1:-1]
    try:
        return int(v)
    except ValueError:
        pass
    try:
        return float(low.replace("d", "e"))
    except ValueError:
        return v


def read_control(path: str) -> dict:
    """Every `key = value` of the namelist group(s) in control.fwh (App. A1),
    keys lower-cased; '!' comments are dropped."""
    text = []
    with open(path) as fh:
        for line in fh:
            text.append(line.split("!", 1)[0])
    body = "\n".join(text)
    groups = re.findall(r"&\w+(.*?)/", body, flags=re.S) or [body]
    out = {}
    for g in groups:
        for k, v in _NAMELIST_ITEM.findall(g):
            out[k.lower()] = _nl_value(v)
    return out


def write_control(path: str, values: dict, group: str = "control") -> None:
    with open(path, "w") as fh:
        fh.write(f"&{group}\n")
        for k, v in values.items():
            if isinstance(v, bool):
                s = ".true." if v else ".false."
            elif isinstance(v, str):
                s = f"'{v}'"
            else:
                s = repr(v)
            fh.write(f"  {k} = {s},\n")
        fh.write("/\n")


# --------------------------------------------------------------- geometry ---

def read_surface_geo(path: str) -> SurfaceGeo:
    """FWH_Surface_Geo.dat (App. A2)."""
    with open(path) as fh:
        lines = [ln.strip() for ln in fh if ln.strip()]
    if not lines[0].lower().replace(" ", "").startswith("variables="):
        raise ValueError(f"{path}: first line must be '{GEO_HEADER}'")
    n_faces = int(lines[1].split()[0])
    pos = 2
    faces, rows = [], []
    for f in range(n_faces):
        dims = [int(v) for v in lines[pos].split()[:3]]
        if len(dims) != 3 or min(dims) < 1:
            raise ValueError(f"{path}: Face {f}: bad 'nx ny nz' line {lines[pos]!r}")
        if 1 not in dims:
            raise ValueError(f"{path}: Face {f}: one of nx, ny, nz must be 1 (a block face)")
        pos += 1
        n = dims[0] * dims[1] * dims[2]
        block = np.array([[float(v.replace("D", "E").replace("d", "e")) for v in ln.split()[:7]]
                          for ln in lines[pos:pos + n]], dtype=np.float64)
        if block.shape != (n, 7):
            raise ValueError(f"{path}: Face {f}: expected {n} rows of 7 values")
        pos += n
        faces.append(tuple(dims))
        rows.append(block)
    data = np.concatenate(rows) if rows else np.zeros((0, 7))
    return SurfaceGeo(np.ascontiguousarray(data[:, 0:3]), np.ascontiguousarray(data[:, 3:6]),
                      np.ascontiguousarray(data[:, 6]), faces)


def write_surface_geo(path: str, geo: SurfaceGeo) -> None:
    with open(path, "w") as fh:
        fh.write(GEO_HEADER + "\n")
        fh.write(f"{len(geo.faces)}\n")
        for (nx, ny, nz), (lo, hi) in zip(geo.faces, geo.face_ranges):
            fh.write(f"{nx} {ny} {nz}\n")
            for p in range(lo, hi):
                vals = (*geo.centroids[p], *geo.normals[p], geo.areas[p])
                fh.write(" ".join(f"{v:.17e}" for v in vals) + "\n")


# -------------------------------------------------------------- observers ---

def read_observers(path: str) -> np.ndarray:
    """observers.dat (Sec. III A): [O][3]."""
    rows = []
    with open(path) as fh:
        for ln in fh:
            parts = ln.split()
            if len(parts) >= 3:
                try:
                    rows.append([float(v.replace("D", "E").replace("d", "e")) for v in parts[:3]])
                except ValueError:
                    continue
    return np.asarray(rows, dtype=np.float64).reshape(-1, 3)


def write_observers(path: str, xyz: np.ndarray) -> None:
    with open(path, "w") as fh:
        for x in np.asarray(xyz, dtype=np.float64).reshape(-1, 3):
            fh.write(" ".join(f"{v:.17e}" for v in x) + "\n")


# ----------------------------------------------------------------- frames ---

def frame_path(directory: str, step: int) -> str:
    return os.path.join(directory, f"FWH-{step:08d}.dat")


def read_frame(path: str, n_panels: int, binary: bool) -> np.ndarray:
    """One FWH-xxxxxxxx.dat frame: [5][P] pulsations (rho', u', v', w', p')."""
    if binary:
        size = os.path.getsize(path)
        want = n_panels * 5 * 8
        with open(path, "rb") as fh:
            if size == want:
                raw = fh.read(want)
            elif size == want + 8:  # one Fortran unformatted record
                (n,) = struct.unpack("<i", fh.read(4))
                if n != want:
                    raise ValueError(f"{path}: record of {n} bytes, expected {want}")
                raw = fh.read(want)
            else:
                raise ValueError(f"{path}: {size} bytes, expected {want} (or +8)")
        vals = np.frombuffer(raw, dtype="<f8").reshape(n_panels, 5)
    else:
        rows = []
        with open(path) as fh:
            for ln in fh:
                parts = ln.split()
                if len(parts) < 5:
                    continue
                try:
                    rows.append([float(v.replace("D", "E").replace("d", "e"))
                                 for v in parts[:5]])
                except ValueError:
                    continue  # a header line
        vals = np.asarray(rows, dtype=np.float64)
        if vals.shape != (n_panels, 5):
            raise ValueError(f"{path}: {vals.shape[0]} subface rows, expected {n_panels}")
    return np.ascontiguousarray(vals.T)


def write_frame(path: str, fields_5p: np.ndarray, binary: bool, fortran_record: bool = False):
    f = np.asarray(fields_5p, dtype=np.float64)
    rows = np.ascontiguousarray(f.T)  # [P][5]
    if binary:
        with open(path, "wb") as fh:
            raw = rows.astype("<f8").tobytes()
            if fortran_record:
                fh.write(struct.pack("<i", len(raw)))
            fh.write(raw)
            if fortran_record:
                fh.write(struct.pack("<i", len(raw)))
    else:
        with open(path, "w") as fh:
            fh.write("rho' u' v' w' p'\n")
            for r in rows:
                fh.write(" ".join(f"{v:.17e}" for v in r) + "\n")


def dataset_steps(control: dict) -> list:
    """Iteration steps Kstep_start, Kstep_start + delta_step, ..., Kstep_end."""
    k0 = int(control["kstep_start"])
    k1 = int(control["kstep_end"])
    dk = int(control.get("delta_step", 1))
    if dk < 1 or k1 < k0:
        raise ValueError("need Kstep_end >= Kstep_start and delta_step >= 1")
    return list(range(k0, k1 + 1, dk))


def load_dataset(directory: str, steps, n_panels: int, binary: bool, dtype=np.float32,
                 pinned: bool = False):
    """The frames of `steps` as fields [nt][5][P] in `dtype` (a torch tensor in
    pinned host memory if `pinned`, else a numpy array); the next frame is
    read on a thread while the current one is stored."""
    nt = len(steps)
    if pinned:
        import torch
        tdt = torch.float32 if np.dtype(dtype) == np.float32 else torch.float64
        out_t = torch.empty((nt, 5, n_panels), dtype=tdt).pin_memory()
        out = out_t.numpy()
    else:
        out = np.empty((nt, 5, n_panels), dtype=dtype)
    with ThreadPoolExecutor(max_workers=1) as ex:
        fut = ex.submit(read_frame, frame_path(directory, steps[0]), n_panels, binary) if nt else None
        for i in range(nt):
            frame = fut.result()
            if i + 1 < nt:
                fut = ex.submit(read_frame, frame_path(directory, steps[i + 1]), n_panels, binary)
            out[i] = frame
    return out_t if pinned else out
