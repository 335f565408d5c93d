"""C ABI checks that need no GPU: the library builds, loads and exports
every entry point that include/kf.h declares; the binding has the same names."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(kf_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["kf_create", "kf_destroy", "kf_load_hits", "kf_load_seeds", "kf_set_alignment",
              "kf_find_tracks", "kf_remove_duplicates", "kf_fit_tracks", "kf_fit_adjoint",
              "kf_get_tracks", "kf_get_fit", "kf_capture_graph", "kf_launch_graph", "kf_autotune",
              "kf_get_counters", "kf_sync", "kf_last_error"]:
        assert n in names, n


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_1906_11744_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    from paper_1906_11744_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_host_argument_errors_without_gpu():
    """kf_create rejects bad geometry and settings before touching the device."""
    import ctypes

    from paper_1906_11744_gb300 import _lib, make_config, make_detector
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    bad_det = make_detector([10.0, 5.0], [0.02, 0.02])  # radii must increase
    assert lib.kf_create(ctypes.byref(bad_det), ctypes.byref(make_config()), ctypes.byref(ctx)) == _lib.KF_ERR_ARG
    det = make_detector([5.0, 10.0], [0.02, 0.02])
    for cfg in (make_config(max_cands=0), make_config(max_cands=17), make_config(lanes_per_seed=5),
                make_config(lanes_per_seed=4, max_cands=6), make_config(block_threads=48),
                make_config(find_regcap=1, block_threads=256), make_config(find_regcap=2),
                make_config(chi2_cut=-1.0)):
        assert lib.kf_create(ctypes.byref(det), ctypes.byref(cfg), ctypes.byref(ctx)) == _lib.KF_ERR_ARG


def test_duplicate_cut_argument_errors_without_gpu():
    """Seed-cleaning and duplicate pre-cut settings are checked before the device:
    negative or non-finite cuts, an eta window of seed cleaning outside
    (0, KF_SEED_MAX_DETA], more than three shared seed hits.  Valid settings get
    past the checks (and fail only at the device, absent here)."""
    import ctypes
    import math

    from paper_1906_11744_gb300 import _lib, make_config, make_detector
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    det = make_detector([5.0, 10.0], [0.02, 0.02])
    bad = (make_config(dup_deta=-0.1), make_config(dup_dphi=math.inf), make_config(dup_dpt=math.nan),
           make_config(seed_clean=2), make_config(seed_clean=1, seed_deta=0.0),
           make_config(seed_clean=1, seed_deta=1.5), make_config(seed_clean=1, seed_dphi=-1.0),
           make_config(seed_clean=1, seed_dpt=math.inf), make_config(seed_clean=1, seed_min_shared=4),
           make_config(seed_clean=1, seed_min_shared=-1))
    for cfg in bad:
        assert lib.kf_create(ctypes.byref(det), ctypes.byref(cfg), ctypes.byref(ctx)) == _lib.KF_ERR_ARG
    ok = (make_config(dup_deta=0.02, dup_dphi=0.02, dup_dpt=0.3),
          make_config(seed_clean=1, seed_deta=_lib.KF_SEED_MAX_DETA, seed_min_shared=3),
          make_config(seed_clean=0, seed_deta=0.0))  # cuts of a disabled cleaning are not checked
    for cfg in ok:
        rc = lib.kf_create(ctypes.byref(det), ctypes.byref(cfg), ctypes.byref(ctx))
        assert rc != _lib.KF_ERR_ARG
        if rc == _lib.KF_OK:
            lib.kf_destroy(ctx)


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1906_11744_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(_lib.KFError):
        _lib.load()


def test_detector_struct_layout_matches_the_header(tmp_path):
    """The binding's kf_detector has the header's size and field offsets
    (a C program compiled against include/kf.h prints them)."""
    import ctypes
    import shutil
    import subprocess

    from paper_1906_11744_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in _lib.kf_detector._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "kf.h"\nint main(void) {\n'
                    '  printf("size %zu\\n", sizeof(kf_detector));\n' +
                    "".join(f'  printf("{f} %zu\\n", offsetof(kf_detector, {f}));\n' for f in fields) +
                    "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(_lib.kf_detector)
    for f in fields:
        assert int(out[f]) == getattr(_lib.kf_detector, f).offset, f


def test_disk_geometry_argument_errors_without_gpu():
    """kf_create rejects a bad endcap geometry before touching the device:
    too many disks, disk planes not increasing in |z| or at z <= 0, radii out
    of order, a non-positive radial resolution or eta_barrel, a negative
    thickness or loss, and a field factor outside [0.2, 5] over the disks'
    reach."""
    import ctypes

    from paper_1906_11744_gb300 import _lib, make_config, make_detector
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    good = dict(disk_z=(130.0, 150.0), disk_rmin=15.0, disk_rmax=110.0, disk_x0=0.02, disk_eloss=0.0,
                sigma_r=0.1, eta_barrel=0.9)
    too_many = make_detector([5.0, 10.0], [0.02, 0.02], **good)
    too_many.n_disks = 17  # beyond KF_MAX_DISKS (the binding refuses to build such a detector)
    assert lib.kf_create(ctypes.byref(too_many), ctypes.byref(make_config()), ctypes.byref(ctx)) == _lib.KF_ERR_ARG
    with pytest.raises(ValueError):
        make_detector([5.0, 10.0], [0.02, 0.02], disk_z=tuple(130.0 + 10 * k for k in range(17)))
    bad = [dict(disk_z=(150.0, 130.0)),
           dict(disk_z=(-130.0, 150.0)), dict(disk_rmin=110.0, disk_rmax=15.0), dict(disk_rmin=0.0),
           dict(sigma_r=0.0), dict(eta_barrel=0.0), dict(disk_x0=-0.01), dict(disk_eloss=-1e-3),
           dict(disk_z=(130.0, 1000.0))]
    for b in bad:
        kw = {**good, **b}
        field = dict(field_cz=-1.0e-6) if b.get("disk_z") == (130.0, 1000.0) else {}
        det = make_detector([5.0, 10.0], [0.02, 0.02], **field, **kw)
        assert lib.kf_create(ctypes.byref(det), ctypes.byref(make_config()), ctypes.byref(ctx)) == _lib.KF_ERR_ARG, b
