"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/abd.h (no compute call: no GPU needed)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "abd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(abd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in ("abd_scene_create", "abd_partition", "abd_step", "abd_state_get"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2605_15875_gb300 import abd, build
    build.build()
    L = abd.load()
    names = _declared()
    assert sorted(abd.EXPORTS) == names
    for n in names:
        assert hasattr(L, n), n


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2605_15875_gb300 import abd
    with pytest.raises(RuntimeError):
        abd.load(str(tmp_path / "missing.so"))


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2605_15875_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "abd_oracle" not in txt, f


def test_oracle_shares_no_code_with_the_library():
    """The oracle includes only its own header and the C library, and its
    Python wrapper imports nothing from the product package."""
    odir = os.path.join(ROOT, "oracle")
    c = open(os.path.join(odir, "abd_oracle.c")).read() + open(os.path.join(odir, "abd_oracle.h")).read()
    includes = set(re.findall(r'#include\s*[<"]([^>"]+)[>"]', c))
    assert includes <= {"abd_oracle.h", "math.h", "stdio.h", "stdlib.h", "string.h", "stdint.h"}, includes
    py = open(os.path.join(odir, "__init__.py")).read()
    assert "paper_2605_15875_gb300" not in py and "libabd.so" not in py


def test_ctypes_struct_layouts_match_the_header(tmp_path):
    """Sizes of the ABI structs as gcc lays them out from include/abd.h equal
    the ctypes mirrors used by the binding."""
    import ctypes
    import subprocess
    from paper_2605_15875_gb300 import abd
    names = ["abd_scene_desc", "abd_partition_desc", "abd_step_params", "abd_step_stats", "abd_server_desc",
             "abd_request_info"]
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "abd.h"\nint main(void){\n' +
                   "".join(f'printf("%zu\\n", sizeof({n}));\n' for n in names) + "return 0;}\n")
    exe = tmp_path / "sz"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    mirrors = [abd.SceneDesc, abd.PartitionDesc, abd.StepParams, abd.StepStats, abd.ServerDesc, abd.RequestInfo]
    assert got == [ctypes.sizeof(m) for m in mirrors]


def test_server_and_partition_calls_reject_bad_arguments():
    """Argument checks of the serving and partition calls happen before any
    device work, so they answer on a machine without a GPU."""
    import ctypes
    from paper_2605_15875_gb300 import abd, build
    build.build()
    L = abd.load()
    h = ctypes.c_void_p()
    bad = abd.ServerDesc(device=0, n_streams=0, hbm_budget_bytes=0)
    assert L.abd_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = abd.ServerDesc(device=0, n_streams=2, hbm_budget_bytes=-5)
    assert L.abd_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    t = ctypes.c_int64()
    assert L.abd_server_submit(None, None, None, None, 1, ctypes.byref(t)) == -1
    assert L.abd_server_submit_keyed(None, 1, None, None, None, 1, ctypes.byref(t)) == -1
    assert L.abd_server_release(None, 1) == -1
    assert L.abd_scene_broadphase(None, 2) == -1
    n = ctypes.c_int32()
    assert L.abd_partition_planes(None, None, 0, ctypes.byref(n)) == -1
    assert L.abd_pd_update(0, None, None, 0.0, 0.0, None, None) == -1


def test_every_status_code_has_its_own_text_and_null_arguments_are_rejected():
    """Each status the header enumerates maps to a distinct message; calls
    given NULL handles fail with ABD_E_INVALID before any device work."""
    import ctypes
    import re
    from paper_2605_15875_gb300 import abd, build
    build.build()
    L = abd.load()
    hdr = open(os.path.join(ROOT, "include", "abd.h")).read()
    codes = {int(v) for v in re.findall(r"ABD_(?:E_)?[A-Z_]+ = (-?\d+),?\s*(?:/\*[^*]*\*/)?\s*\n", hdr[hdr.index("ABD_OK = 0"):])}
    codes.add(0)
    assert {0, 1, 2, 3, 4, -1, -2, -3, -4, -5, -6, -7} <= codes
    texts = {c: L.abd_status_string(c).decode() for c in codes}
    assert len(set(texts.values())) == len(codes) and "unknown status" not in texts.values()
    assert L.abd_status_string(12345).decode() == "unknown status"
    st = abd.StepStats()
    p = abd.default_params()
    assert L.abd_step(None, ctypes.byref(p), ctypes.byref(st)) == -1
    assert L.abd_state_get(None, None, None, 0) == -1
    assert L.abd_candidates_noalloc(None, None, None, 1e-3, None, 0, None) == -1


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    """A C program built with gcc against include/abd.h links libabd.so and
    calls its host-only entry points (no GPU needed): default parameters, the
    load-balancing law, status texts, and an argument check."""
    import subprocess
    from paper_2605_15875_gb300 import build
    lib = build.build()
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "abd.h"
int main(void) {
    abd_step_params p = abd_step_params_default();
    double tau[3] = {3.0, 1.0, 1.0}, delta[2], T[2];
    int rc = abd_pd_update(3, tau, NULL, 0.5, 0.0, delta, T);
    printf("%g %g %d %d\n", p.h, p.dhat, p.max_admm, rc);
    printf("%.17g %.17g %.17g %.17g\n", T[0], T[1], delta[0], delta[1]);
    printf("%s|%s\n", abd_status_string(ABD_OK), abd_status_string(ABD_E_PENETRATION));
    printf("%d\n", abd_step(NULL, &p, NULL));
    return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-labd", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.splitlines()
    assert lines[0].split() == ["0.01", "0.001", "200", "0"]
    T0, T1, d0, d1 = map(float, lines[1].split())
    assert T0 == 0.5 and T1 == 0.0  # (3 - 1) / (3 + 1), (1 - 1) / (1 + 1)
    assert d0 == -0.25 and d1 == 0.0  # -(kp T): the plane moves toward the slower slab
    assert lines[2] == "ok|penetration detected"
    assert lines[3] == "-1"


def test_batched_world_rejects_mismatched_scenes_before_device_work():
    """abd_scene_create_batch checks its scenes before any device work: one
    set of ground planes and one gravity for the whole world, 1..256 scenes;
    the layout and Newton queries reject NULL handles."""
    import ctypes
    from paper_2605_15875_gb300 import abd, build, scenes
    build.build()
    L = abd.load()
    a = scenes.random_pile(1, 8, levels=(1,))
    b = scenes.cube_stack(ground=False)
    descs = (abd.SceneDesc * 2)(abd.scene_desc(a), abd.scene_desc(b))
    h = ctypes.c_void_p()
    assert L.abd_scene_create_batch(ctypes.cast(descs, ctypes.c_void_p), 2, None, ctypes.byref(h)) == -1
    c = scenes.random_pile(2, 8, levels=(1,))
    c.gravity = np.array([0.0, -1.0, 0.0])
    descs = (abd.SceneDesc * 2)(abd.scene_desc(a), abd.scene_desc(c))
    assert L.abd_scene_create_batch(ctypes.cast(descs, ctypes.c_void_p), 2, None, ctypes.byref(h)) == -1
    assert L.abd_scene_create_batch(ctypes.cast(descs, ctypes.c_void_p), 0, None, ctypes.byref(h)) == -1
    assert L.abd_scene_create_batch(ctypes.cast(descs, ctypes.c_void_p), 257, None, ctypes.byref(h)) == -1
    n = ctypes.c_int32()
    assert L.abd_batch_layout(None, None, 0, ctypes.byref(n)) == -1
    assert L.abd_partition_newton(None, None, 0, ctypes.byref(n)) == -1
    assert L.abd_scene_reserve(None, 16) == -1
