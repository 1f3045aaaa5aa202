"""The C ABI library builds, loads and answers its host-only calls (no GPU).

Checks that libmg.so exports every function include/mg.h, include/mg_box.h
and include/unet.h declare, that the
multigrid level sizes it computes agree with the oracle's for many sizes,
and that argument validation happens on the host before any CUDA call.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mg():
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg as M
    return M


def _declared(headers=("mg.h", "mg_box.h", "unet.h")):
    names = set()
    for hdr in headers:
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(mg):
    names = _declared()
    assert "mg_create_hierarchy" in names and "mg_solve" in names and len(names) >= 10
    lib = C.CDLL(mg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi(mg):
    from paper_2001_02327_gb300 import unet as U
    for n in _declared():
        assert hasattr(mg, n) or hasattr(U, n), n


def test_default_options(mg):
    o = mg.mg_default_options()
    assert (o.nu_pre, o.nu_post, o.max_cycles, o.rel_tol) == (2, 1, 50, 1e-10)
    assert o.precision == mg.MG_FP64 and o.guess == mg.MG_GUESS_INTERP and o.force_stencil == mg.MG_FORCE_EQ2


def test_level_sizes_match_oracle(mg, oracle):
    for M in list(range(2, 600)) + [1026, 2050, 4098]:
        assert mg.mg_level_sizes(M) == oracle.mg_sizes(M), M


def test_status_strings(mg):
    for s in range(8):
        assert mg.mg_status_str(s).startswith("MG_")


def _desc(mg, **kw):
    from paper_2001_02327_gb300 import inputs as I
    H = I.config_3d_offset_sphere(n=16, levels=2)
    d = mg.desc_from(H)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", ["dim", "levels", "n_odd", "offset", "h0", "opt", "interface", "stop",
                                 "stop_frozen", "parent", "tree_flag"])
def test_invalid_arguments_rejected_on_host(mg, bad):
    d = _desc(mg)
    opt = None
    if bad == "dim":
        d.dim = 4
    elif bad == "levels":
        d.num_levels = 9
    elif bad == "n_odd":
        d.n[1] = 15
    elif bad == "offset":
        d.lo[1][0] = d.lo[0][0]           # offset 0 parent cells: buffer would leave the parent
    elif bad == "h0":
        d.h0 = -1.0
    elif bad == "opt":
        opt = mg.options(nu_pre=0, nu_post=0)
    elif bad == "interface":
        opt = mg.options(interface=2)
    elif bad == "stop":
        opt = mg.options(stop=2)
    elif bad == "parent":
        d.tree = 1
        d.parent[1] = 1                   # a patch cannot be its own parent
    elif bad == "tree_flag":
        d.tree = 2
    elif bad == "stop_frozen":
        # the force-change test is defined on the buffer-ring method only
        opt = mg.options(stop=mg.MG_STOP_FORCE, interface=mg.MG_IFACE_FROZEN)
    with pytest.raises(mg.MGError) as e:
        mg.mg_create_hierarchy([d], opt)
    assert e.value.status == mg.MG_EINVAL
    assert mg.mg_error_message(None)


def _box_desc(mg, **kw):
    from paper_2001_02327_gb300 import inputs as I
    return mg.box_desc_from(I.box_3d_sphere(n=(24, 32, 16), levels=3))


@pytest.mark.parametrize("bad", ["dim", "patches", "n_odd", "n_small", "offset", "off_grid", "h0", "parent",
                                 "frozen", "force_stop", "user_guess", "learned_guess", "inner_max"])
def test_box_invalid_arguments_rejected_on_host(mg, bad):
    d = _box_desc(mg)
    opt = None
    if bad == "dim":
        d.dim = 1
    elif bad == "patches":
        d.num_patches = 0
    elif bad == "n_odd":
        d.n[1][2] = 15
    elif bad == "n_small":
        d.n[0][1] = 1
    elif bad == "offset":
        d.lo[1][1] = d.lo[0][1]             # offset 0 parent cells along y
    elif bad == "off_grid":
        d.lo[2][0] += 0.3 * d.h0            # not on a parent cell face
    elif bad == "h0":
        d.h0 = 0.0
    elif bad == "parent":
        d.tree = 1
        d.parent[2] = 2
    elif bad == "frozen":
        opt = mg.options(interface=mg.MG_IFACE_FROZEN)
    elif bad == "force_stop":
        opt = mg.options(stop=mg.MG_STOP_FORCE)
    elif bad == "user_guess":
        opt = mg.options(guess=mg.MG_GUESS_USER)
    elif bad == "learned_guess":
        opt = mg.options(guess=mg.MG_GUESS_LEARNED)
    elif bad == "inner_max":
        opt = mg.options(precision=mg.MG_MIXED, inner_max=99)
    with pytest.raises(mg.MGError) as e:
        mg.mg_box_create(d, opt)
    assert e.value.status == mg.MG_EINVAL
    assert mg.mg_box_error_message(None)


def test_null_handles(mg):
    assert mg.LIB.mg_box_destroy(None) == mg.MG_OK
    assert mg.LIB.mg_box_solve(None, None) == mg.MG_EINVAL
    assert mg.LIB.mg_box_forces(None, 0, None, None) == mg.MG_EINVAL
    assert mg.LIB.mg_box_set_density(None, 0, None, None, None) == mg.MG_EINVAL
    assert mg.LIB.mg_box_level_sizes(None, 0, None, 0) == -1
    assert mg.LIB.mg_destroy(None) == mg.MG_OK
    assert mg.LIB.mg_solve(None, None) == mg.MG_EINVAL
    assert mg.LIB.mg_forces(None, 0, 0, None, None) == mg.MG_EINVAL
    assert mg.LIB.mg_set_density(None, 0, 0, None, None, None) == mg.MG_EINVAL
    assert mg.LIB.mg_default_options(None) == mg.MG_EINVAL


def test_product_path_does_not_touch_the_oracle():
    """No file of the package or the C sources refers to the oracle."""
    pkg = os.path.join(ROOT, "paper_2001_02327_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f
