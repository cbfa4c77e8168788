"""Input files of OpenCFD-FWH (Sec. III A, App. A): readers against their
writers and hand-written files (CPU only).

FWH_Surface_Geo.dat follows App. A2 line by line; control.fwh is a Fortran
namelist (App. A1); the per-frame dataset files follow the reading stated in
paper_2312_16263_gb300/fwh_io.py (App. A3's figure is missing).  The Faces
read from the geometry feed the Face partition of Sec. III A.
"""
import numpy as np
import pytest

from paper_2312_16263_gb300 import fwh_io
from paper_2312_16263_gb300.shard import partition_faces


def _geo():
    rng = np.random.default_rng(4)
    faces = [(3, 4, 1), (1, 5, 2), (6, 1, 1)]
    P = sum(a * b * c for a, b, c in faces)
    y = rng.normal(size=(P, 3))
    n = rng.normal(size=(P, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return fwh_io.SurfaceGeo(y, n, rng.uniform(0.1, 1.0, P), faces)


def test_surface_geo_round_trip(tmp_path):
    g = _geo()
    path = tmp_path / "FWH_Surface_Geo.dat"
    fwh_io.write_surface_geo(str(path), g)
    lines = path.read_text().splitlines()
    assert lines[0] == "variables=x,y,z,n1,n2,n3,dS" and lines[1] == "3" and lines[2] == "3 4 1"
    r = fwh_io.read_surface_geo(str(path))
    np.testing.assert_array_equal(r.centroids, g.centroids)
    np.testing.assert_array_equal(r.normals, g.normals)
    np.testing.assert_array_equal(r.areas, g.areas)
    assert r.faces == g.faces and r.face_sizes == [12, 10, 6]
    assert r.face_ranges == [(0, 12), (12, 22), (22, 28)]
    assert partition_faces(r.face_sizes, 2) == [[0], [1, 2]]


def test_surface_geo_hand_written_and_errors(tmp_path):
    path = tmp_path / "g.dat"
    path.write_text("variables=x,y,z,n1,n2,n3,dS\n1\n2 1 1\n"
                    "0 0 1 0 0 1 0.5D0\n1.5d0 0 1 0 0 1 0.25\n")
    r = fwh_io.read_surface_geo(str(path))
    np.testing.assert_array_equal(r.areas, [0.5, 0.25])
    assert r.centroids[1, 0] == 1.5
    path.write_text("variables=x,y,z,n1,n2,n3,dS\n1\n2 2 2\n")
    with pytest.raises(ValueError):
        fwh_io.read_surface_geo(str(path))


def test_control_namelist(tmp_path):
    path = tmp_path / "control.fwh"
    path.write_text("&control_para\n Kstep_start = 1000, Kstep_end = 1200 ! frames\n"
                    " delta_step = 10, FWH_data_Format = 0,\n Mach = 0.17, AoA = 5.5d0,\n"
                    " dt = 1.0E-5, use_mpi = .true., name = 'case'\n/\n")
    c = fwh_io.read_control(str(path))
    assert c["kstep_start"] == 1000 and c["kstep_end"] == 1200 and c["delta_step"] == 10
    assert c["fwh_data_format"] == 0 and c["mach"] == 0.17 and c["aoa"] == 5.5
    assert c["dt"] == 1e-5 and c["use_mpi"] is True and c["name"] == "case"
    assert fwh_io.dataset_steps(c) == list(range(1000, 1201, 10))
    out = tmp_path / "c2.fwh"
    fwh_io.write_control(str(out), {"Kstep_start": 3, "Kstep_end": 7, "delta_step": 2})
    assert fwh_io.dataset_steps(fwh_io.read_control(str(out))) == [3, 5, 7]


def test_observers_file(tmp_path):
    xyz = np.random.default_rng(1).normal(size=(5, 3)) * 100
    path = tmp_path / "observers.dat"
    fwh_io.write_observers(str(path), xyz)
    np.testing.assert_array_equal(fwh_io.read_observers(str(path)), xyz)


@pytest.mark.parametrize("binary,record", [(True, False), (True, True), (False, False)])
def test_dataset_frames_to_field_layout(tmp_path, binary, record):
    rng = np.random.default_rng(2)
    P, steps = 28, [100, 110, 120, 130]
    frames = [rng.normal(size=(5, P)) for _ in steps]
    for s, f in zip(steps, frames):
        fwh_io.write_frame(fwh_io.frame_path(str(tmp_path), s), f, binary, record)
    got = fwh_io.load_dataset(str(tmp_path), steps, P, binary, dtype=np.float64)
    assert got.shape == (4, 5, P)
    np.testing.assert_array_equal(got, np.stack(frames))
    got32 = fwh_io.load_dataset(str(tmp_path), steps, P, binary, dtype=np.float32)
    np.testing.assert_array_equal(got32, np.stack(frames).astype(np.float32))
    with pytest.raises(ValueError):
        fwh_io.read_frame(fwh_io.frame_path(str(tmp_path), 100), P + 1, binary)
