"""The C-ABI library loads and exports every symbol include/ff.h declares.

CPU only: no compute call is made (there may be no GPU here).
"""
from __future__ import annotations

import ctypes as ct
import os
import re

from paper_1703_02563_gb300 import ff

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared() -> list[str]:
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ff_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ff_create", "ff_features", "ff_match", "ff_filter", "ff_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ff.lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(ff.EXPORTED) == _declared()


def test_library_is_built_for_sm_103a():
    from paper_1703_02563_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_host_side_argument_checks_need_no_gpu():
    lib = ff.lib()
    c = ff.ff_config()
    assert lib.ff_config_default(ct.byref(c)) == ff.FF_OK
    assert (c.patch, c.n_coeffs, c.seed_leaf) == (8, 9, 8)
    assert lib.ff_config_default(None) == ff.FF_EINVAL
    assert lib.ff_features(None, 0, None, 1, 1, 1) == ff.FF_EINVAL
    assert lib.ff_match(None, 0, 0, None, None, None) == ff.FF_EINVAL
    assert lib.ff_filter(None, None, None, None) == ff.FF_EINVAL
    assert lib.ff_sync(None) == ff.FF_EINVAL
    assert ff.status_string(ff.FF_ETIMEOUT) == "FF_ETIMEOUT"
    out = ct.c_void_p()
    bad = ff.Config(channels=2).c()
    assert lib.ff_create(ct.byref(bad), 0, None, ct.byref(out)) == ff.FF_EINVAL
    bad = ff.Config(seed_leaf=9).c()
    assert lib.ff_create(ct.byref(bad), 0, None, ct.byref(out)) == ff.FF_EINVAL
    bad = ff.Config(max_width=5000).c()
    assert lib.ff_create(ct.byref(bad), 0, None, ct.byref(out)) == ff.FF_EINVAL
    lib.ff_destroy(None)


def test_server_admission_by_memory_needs_no_gpu():
    cfg = ff.Config(channels=3, scales=4, iters=6, max_width=1024, max_height=436)
    per = ff.ff_slot_bytes(cfg)
    # the features alone: 2 frames x 4 levels of 32-byte vectors
    assert per > 2 * 1024 * 436 * 32
    big = ff.Config(channels=3, scales=4, iters=6, max_width=1920, max_height=1080)
    assert ff.ff_slot_bytes(big) > 4 * per
    # a budget below one slot is refused before any device call
    out = ct.c_void_p()
    c = cfg.c()
    assert ff.lib().ff_server_create(ct.byref(c), 0, per - 1, 8, ct.byref(out)) == ff.FF_ENOMEM
    assert out.value is None


def test_config_limits_are_checked_before_any_device_call():
    out = ct.c_void_p()
    for field, value in (("max_width", 4097), ("max_height", 0), ("scales", 9), ("iters", 65),
                         ("schedule", 4), ("channels", 2)):
        c = ff.Config(**{field: value}).c()
        assert ff.lib().ff_create(ct.byref(c), 0, None, ct.byref(out)) == ff.FF_EINVAL, field
        assert out.value is None
