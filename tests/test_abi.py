"""The C-ABI library builds for sm_103a, loads on the host and exports every
entry point declared in include/*.h; host-side argument checks reject bad
calls before touching a device.  No kernel is launched here."""
import ctypes
import os
import re

import pytest

import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import _build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ms_\w+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    # the Python binding wraps exactly the declared set
    bound = {s[0] for s in msgs._SIGNATURES}
    assert bound == set(names)
    assert lib.ms_version() == 100


def test_workspace_sizes():
    ws = msgs.ms_bin_workspace_bytes(1_000_000, 4108, 8_000_000)
    assert ws > 4 * 4 * 1_000_000 + 4 * 4 * 8_000_000
    assert msgs.ms_bin_workspace_bytes(10, 1, 1) > 0
    assert msgs.ms_bin_workspace_bytes(10, 0, 1) == 0          # no tiles
    assert msgs.ms_bin_workspace_bytes(10, 1, 0) == 0          # no capacity
    assert msgs.ms_bin_workspace_bytes(10, 1, 1 << 31) == 0    # capacity > 2^30
    assert msgs.ms_bin_workspace_bytes(-1, 1, 1) == 0
    # the raster workspace holds, besides the segment states, one half-row
    # mask word per tile-list entry for the list kernel
    a = msgs.ms_raster_workspace_bytes(260, 1_000_000)
    b = msgs.ms_raster_workspace_bytes(260, 2_000_000)
    assert a > 4 * 1_000_000 and b - a >= 4 * 1_000_000
    assert msgs.ms_raster_workspace_bytes(0, 1) == 0
    assert msgs.ms_raster_workspace_bytes(65537, 1) == 0
    assert msgs.ms_raster_workspace_bytes(1, 1 << 30) == 0


def test_argument_errors_need_no_device():
    lib = msgs.lib()
    cam = msgs.camera_struct(inputs.config1_camera())
    proj = msgs.ms_proj_t()
    # NULL scene
    assert lib.ms_project(None, ctypes.byref(cam), 0, ctypes.byref(proj), None) == msgs.MS_ERR_INVALID_ARG
    assert b"scene" in lib.ms_last_error()
    sc = msgs.ms_scene_t()
    sc.n = -5
    assert lib.ms_scene_prepare(ctypes.byref(sc), None) == msgs.MS_ERR_INVALID_ARG
    sc.n = 10
    assert lib.ms_project(ctypes.byref(sc), ctypes.byref(cam), 0, ctypes.byref(proj), None) == msgs.MS_ERR_INVALID_ARG
    # ms_project_views: the view count and the arrays are checked first
    empty = msgs.ms_scene_t()
    cams2 = (msgs.ms_camera_t * 2)(cam, cam)
    projs2 = (msgs.ms_proj_t * 2)(proj, proj)
    for n_views in (0, -1, msgs.MS_MAX_PROJ_VIEWS + 1):
        assert lib.ms_project_views(ctypes.byref(empty), cams2, n_views, 0, projs2,
                                    None) == msgs.MS_ERR_INVALID_ARG
        assert b"n_views" in lib.ms_last_error()
    assert lib.ms_project_views(ctypes.byref(empty), None, 1, 0, projs2, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_project_views(ctypes.byref(empty), cams2, 1, 0, None, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_project_views(ctypes.byref(empty), cams2, 2, 7, projs2, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_project_views(ctypes.byref(empty), cams2, 2, 0, projs2,
                                None) == msgs.MS_ERR_INVALID_ARG  # NULL output buffers
    assert b"NULL" in lib.ms_last_error()
    # bad camera
    bad = msgs.camera_struct(inputs.config1_camera())
    bad.width = 0
    assert lib.ms_update_range(ctypes.byref(sc), ctypes.byref(bad), 1, None) == msgs.MS_ERR_INVALID_ARG
    # ms_bin without workspace
    bins = msgs.ms_bins_t()
    bins.dup_capacity = 16
    assert lib.ms_bin(ctypes.byref(proj), 10, ctypes.byref(cam), ctypes.byref(bins), None, 0, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_raster(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(cam), None, None, None, None, None, 0, None) == msgs.MS_ERR_INVALID_ARG
    assert msgs.ms_raster_workspace_bytes(4108, 1 << 20) > 0
    assert msgs.ms_raster_workspace_bytes(0, 1 << 20) == 0
    # ms_raster_ex: an unknown strategy is rejected before anything else
    fake = 1 << 20
    fproj = msgs.ms_proj_t(fake, fake, fake, fake, 0, 0, fake, 10)
    fbins = msgs.ms_bins_t(fake, fake, fake, 16)
    for strategy in (-1, 6, 1000):
        assert lib.ms_raster_ex(ctypes.byref(fproj), ctypes.byref(fbins), ctypes.byref(cam), fake,
                                None, None, None, fake, 1 << 30, strategy,
                                None) == msgs.MS_ERR_INVALID_ARG
        assert b"strategy" in lib.ms_last_error()
    for strategy in msgs.STRATEGIES.values():  # then the usual argument checks
        assert lib.ms_raster_ex(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(cam), None,
                                None, None, None, None, 0, strategy,
                                None) == msgs.MS_ERR_INVALID_ARG


def test_multi_view_helpers_check_lengths_first():
    """The view helpers reject mismatched lists before touching a device."""
    cam = msgs.camera_struct(inputs.config1_camera())
    with pytest.raises(msgs.MsError):
        msgs.ms_project_views(msgs.ms_scene_t(), [cam, cam], msgs.MS_SELECTIVE,
                              [msgs.ms_proj_t()])
    with pytest.raises(msgs.MsError):
        msgs.render_views(None, [object()], [], "selective")
    with pytest.raises(msgs.MsError):
        msgs.render_views(None, [object()], [object()], "selective", streams=[])


def test_backward_argument_errors_need_no_device():
    lib = msgs.lib()
    cam = msgs.camera_struct(inputs.config1_camera())
    fake = 1 << 20                      # never dereferenced: the checks fail first
    sc = msgs.ms_scene_t(10, 1, -1, *([fake] * 10))
    proj = msgs.ms_proj_t(fake, fake, fake, fake, 0, 0, fake, 10)
    bins = msgs.ms_bins_t(fake, fake, fake, 16)
    grads = msgs.ms_grads_t(*([fake] * 5))
    ws = msgs.ms_raster_bwd_workspace_bytes(10)
    assert ws >= 10 * 9 * 4 + 4 and ws % 256 == 0
    assert msgs.ms_raster_bwd_views_workspace_bytes(10, 1) == ws
    assert msgs.ms_raster_bwd_views_workspace_bytes(10, 3) > ws
    assert msgs.ms_raster_bwd_views_workspace_bytes(10, 0) == 0
    assert msgs.ms_raster_bwd_views_workspace_bytes(10, msgs.MS_MAX_BWD_VIEWS + 1) == 0
    assert msgs.ms_raster_bwd_workspace_bytes(-1) == 0
    rws = msgs.ms_raster_workspace_bytes(cam.width // 16 * (cam.height // 16), 16)

    def bwd(flags, ws_bytes=ws, g=grads, s=sc, rws_bytes=rws):
        return lib.ms_raster_bwd(ctypes.byref(s), ctypes.byref(cam), ctypes.byref(proj),
                                 ctypes.byref(bins), fake, fake, fake, rws_bytes, fake,
                                 ctypes.byref(g), flags, fake, ws_bytes, None)
    assert bwd(8) == msgs.MS_ERR_INVALID_ARG and b"flags" in lib.ms_last_error()
    assert bwd(msgs.MS_BWD_ACCUMULATE, ws - 4) == msgs.MS_ERR_INVALID_ARG
    assert bwd(0, g=msgs.ms_grads_t(fake, fake, 0, fake, fake)) == msgs.MS_ERR_INVALID_ARG
    bad_deg = msgs.ms_scene_t(10, 1, 4, *([fake] * 10))
    assert bwd(0, s=bad_deg) == msgs.MS_ERR_INVALID_ARG
    assert bwd(0, rws_bytes=rws - 16) == msgs.MS_ERR_INVALID_ARG
    assert b"raster workspace" in lib.ms_last_error()
    v = msgs.bwd_view(cam, proj, bins, fake, fake, fake, rws, fake)
    arr = (msgs.ms_bwd_view_t * 1)(v)
    assert lib.ms_raster_bwd_views(ctypes.byref(sc), arr, 0, ctypes.byref(grads), 0, fake, ws,
                                   None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_raster_bwd_views(ctypes.byref(sc), arr, 1, ctypes.byref(grads), 0, fake,
                                   ws - 16, None) == msgs.MS_ERR_INVALID_ARG
    # L1 loss: count 0 is a no-op, negative counts, NULL and misaligned buffers fail
    assert lib.ms_l1_loss_grad(None, None, 0, 1.0, None, None, None) == msgs.MS_OK
    assert lib.ms_l1_loss_grad(fake, fake, -1, 1.0, fake, None, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_l1_loss_grad(fake, None, 8, 1.0, fake, None, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_l1_loss_grad(fake + 4, fake, 8, 1.0, fake, None, None) == msgs.MS_ERR_INVALID_ARG


def test_inputs_module_stands_alone():
    """The shared input module (used by both the oracle side and the CUDA
    side) imports nothing but numpy and the standard library, so neither
    side's arithmetic can leak into the other's inputs."""
    import ast
    src = open(os.path.join(ROOT, "paper_2311_17089_gb300", "inputs.py")).read()
    mods = set()
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add((node.module or "").split(".")[0])
    assert mods <= {"numpy", "math", "dataclasses", "__future__"}, mods


def test_product_does_not_reference_oracle():
    pkg = os.path.join(ROOT, "paper_2311_17089_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_serve_argument_errors_need_no_device():
    lib = msgs.lib()
    h = ctypes.c_void_p()

    def create(**kw):
        c = dict(max_gaussians=1000, max_width=256, max_height=256, max_inflight=8, n_streams=2,
                 mem_budget_bytes=1 << 26, initial_capacity=0, device=0)
        c.update(kw)
        cfg = msgs.ms_serve_cfg_t(*c.values())
        return lib.ms_serve_create(ctypes.byref(cfg), ctypes.byref(h))
    for bad in (dict(max_gaussians=0), dict(max_width=0), dict(max_inflight=0),
                dict(n_streams=9), dict(mem_budget_bytes=1000), dict(initial_capacity=-1),
                dict(device=-1)):
        rc = create(**bad)
        assert rc in (msgs.MS_ERR_INVALID_ARG, msgs.MS_ERR_NO_DEVICE), bad
        assert h.value is None
    assert lib.ms_serve_destroy(None) == msgs.MS_OK
    r = msgs.ms_result_t()
    assert lib.ms_serve_poll(None, 1, ctypes.byref(r)) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_serve_submit(None, None, None) == msgs.MS_ERR_INVALID_ARG
    assert lib.ms_serve_clock() > 0.0


def test_shared_sort_argument_errors_need_no_device():
    """The shared depth sort's calls reject bad arguments on the host."""
    lib = msgs.lib()
    fake = 1 << 20                      # never dereferenced: the checks fail first
    E = msgs.MS_ERR_INVALID_ARG
    up = msgs.ms_proj_t(0, 0, fake, fake, 0, 0, fake, 1000)
    assert msgs.ms_sort_depth_workspace_bytes(1000) > 0
    assert msgs.ms_sort_depth_workspace_bytes(-1) == 0
    assert msgs.ms_split_order_workspace_bytes(1000) >= 256
    assert msgs.ms_split_order_workspace_bytes(-1) == 0
    ws = msgs.ms_split_order_workspace_bytes(1000)
    orders = (ctypes.c_void_p * 8)(*([fake] * 8))
    stats = (ctypes.c_void_p * 8)(*([fake] * 8))

    def split(n_views, ws_bytes=ws, o=orders, s=stats, order=fake, n=1000):
        return lib.ms_split_order(ctypes.byref(up), n, order, n_views, o, s, fake, ws_bytes,
                                  None)
    assert split(0) == E and split(9) == E                   # n_views outside 1..8
    assert split(2, ws_bytes=ws - 16) == E                   # workspace too small
    assert split(2, order=None) == E
    assert split(2, n=2000) == E                             # the union holds 1000
    bad = (ctypes.c_void_p * 8)(fake, 0, *([fake] * 6))
    assert split(2, o=bad) == E                              # a NULL view order
    assert lib.ms_sort_depth(ctypes.byref(up), 1000, None, fake, 1 << 30, None) == E
    assert lib.ms_sort_depth(ctypes.byref(up), 1000, fake, fake, 16, None) == E
    cam = msgs.camera_struct(inputs.config1_camera())
    bins = msgs.ms_bins_t(fake, fake, fake, 16)
    assert lib.ms_bin_ordered(ctypes.byref(up), 1000, ctypes.byref(cam), ctypes.byref(bins),
                              None, fake, fake, 1 << 30, None) == E
    sc = msgs.ms_scene_t(10, 1, -1, *([fake] * 10))
    cams = (msgs.ms_camera_t * 2)(cam, cam)
    outs = (msgs.ms_proj_t * 2)(up, up)
    for mask in (0, 4):                                      # none, or a view beyond n_views
        assert lib.ms_project_views_union(ctypes.byref(sc), cams, 2, 0, outs, mask, fake,
                                          fake, None) == E
    assert lib.ms_project_views_union(ctypes.byref(sc), cams, 2, 0, outs, 3, None, fake,
                                      None) == E


def test_depth_order_plan():
    """Frames that list nearly the same Gaussians bin straight from the
    sorted union; frames of very different list sizes get it split."""
    views, split = msgs.depth_order_plan([900, 950, 1000])
    assert views == [0, 1, 2] and not split
    views, split = msgs.depth_order_plan([600_000, 650_000, 34_000])
    assert views == [0, 1, 2] and split
    assert msgs.depth_order_plan([0, 0])[1]                  # nothing listed: split (trivial)
    assert msgs.shared_order_views([614, 649, 417, 34]) == [0, 1]
    assert msgs.shared_order_views([]) == []
