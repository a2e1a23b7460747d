"""CPU-only checks of the boundary: the C ABI library builds for sm_103a,
loads, and exports every function the header declares."""
import ctypes
import os
import subprocess

import pytest


def test_header_declares_expected_calls():
    from paper_1808_09571_gb300 import geo3d
    names = geo3d.declared_functions()
    for n in ("g3d_create", "g3d_destroy", "g3d_get_config", "g3d_set_config",
              "g3d_mesh_load", "g3d_mesh_load_many", "g3d_mesh_build_bvh", "g3d_mesh_build_bvh_many",
              "g3d_mesh_free", "g3d_mesh_free_many", "g3d_mesh_free_many_async", "g3d_mesh_size", "g3d_mesh_export",
              "g3d_distance", "g3d_intersects", "g3d_batch", "g3d_batch_ex", "g3d_batch_hint",
              "g3d_plan_create", "g3d_plan_launch", "g3d_plan_destroy", "g3d_segments", "g3d_volume",
              "g3d_volume_many", "g3d_autotune", "g3d_mlp_num_params", "g3d_mlp_create", "g3d_mlp_destroy",
              "g3d_mlp_set_params", "g3d_mlp_get_params", "g3d_mlp_forward", "g3d_mlp_gradients",
              "g3d_mlp_train_step", "g3d_mlp_train", "g3d_mlp_save", "g3d_mlp_load", "g3d_pair_features",
              "g3d_set_proposal", "g3d_distance_soup_noalloc", "g3d_sync", "g3d_stats_get", "g3d_stats_reset",
              "g3d_profile_begin", "g3d_profile_end", "g3d_debug_words", "g3d_strerror"):
        assert n in names, n


def test_library_builds_and_exports_every_declared_symbol():
    import paper_1808_09571_gb300 as pkg
    from paper_1808_09571_gb300 import geo3d
    path = pkg.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in geo3d.declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)  # loads without a GPU
    lib.g3d_strerror.restype = ctypes.c_char_p
    assert lib.g3d_strerror(-6) == b"candidate list overflow"
    assert lib.g3d_strerror(0) == b"ok"
    assert lib.g3d_strerror(-12) == b"file could not be read or written"
    # every error code the binding knows has its own message
    msgs = {lib.g3d_strerror(code) for code in geo3d.ERRORS}
    assert len(msgs) == len(geo3d.ERRORS) and b"unknown error" not in msgs


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1808_09571_gb300 import geo3d
    with pytest.raises(geo3d.G3DError) as e:
        geo3d.Context(0)
    assert e.value.code == -1


def test_product_path_never_imports_the_oracle():
    root = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1808_09571_gb300")
    for dirpath, _, files in os.walk(root):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f
