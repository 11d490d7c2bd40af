"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point declared in include/rb.h, and its structs
have the layout the Python binding assumes."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1805_06124_gb300 import build as rbbuild
from paper_1805_06124_gb300 import rb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rb_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = rbbuild.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "rb_greedy" in names and "rb_project" in names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_binding(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rb.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rb_options), sizeof(rb_result),'
                   ' offsetof(rb_result, k), offsetof(rb_result, ms_total), offsetof(rb_options, stream),'
                   ' offsetof(rb_options, batched_variant), offsetof(rb_options, timeout_cycles));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(rb.Options), ctypes.sizeof(rb.Result), rb.Result.k.offset,
                    rb.Result.ms_total.offset, rb.Options.stream.offset, rb.Options.batched_variant.offset,
                    rb.Options.timeout_cycles.offset]


def test_default_options(lib):
    L = rb.load()
    o = rb.Options()
    L.rb_default_options(ctypes.byref(o))
    assert o.sweep == rb.SWEEP["df32"] and o.imgs_kappa == 2.0 and o.imgs_max_passes == 4
    assert o.switch_err == 0.0 and o.iters_per_sync >= 1
    assert o.batched_variant == -1 and o.timeout_cycles == 0


def test_bad_options_rejected_before_any_device_call(lib):
    L = rb.load()
    o = rb.Options()
    L.rb_default_options(ctypes.byref(o))
    o.imgs_kappa = 1.0
    h = ctypes.c_void_p()
    assert L.rb_create(ctypes.byref(o), ctypes.byref(h)) == rb.EINVAL
    L.rb_default_options(ctypes.byref(o))
    o.batched_variant = 24
    assert L.rb_create(ctypes.byref(o), ctypes.byref(h)) == rb.EINVAL
    L.rb_default_options(ctypes.byref(o))
    o.switch_err = -1e-6
    assert L.rb_create(ctypes.byref(o), ctypes.byref(h)) == rb.EINVAL
    L.rb_default_options(ctypes.byref(o))
    o.switch_err = float("nan")
    assert L.rb_create(ctypes.byref(o), ctypes.byref(h)) == rb.EINVAL
    L.rb_default_options(ctypes.byref(o))
    o.timeout_cycles = 1000
    assert L.rb_create(ctypes.byref(o), ctypes.byref(h)) == rb.EINVAL
    assert L.rb_greedy(None, None, 1, 1, 1, 0.0, 1, None) == rb.EINVAL
    assert L.rb_project(None, None, 1, 1, 1, None, 1, 1, None, 1) == rb.EINVAL
    k = ctypes.c_int(-1)
    assert L.rb_reconstruct(None, None, 1, 1, 1, None, 1, 1, 0.0, None, 1, None, None, ctypes.byref(k)) == rb.EINVAL
    assert L.rb_eim(None, None, 1, 1, 1, None, None, None, 1, None) == rb.EINVAL
    assert L.rb_greedy_resume(None, None, 1, 1, 1, 0.0, 1, 0, 0, None) == rb.EINVAL
    assert L.rb_trace(None, None, None, None, 0, None) == rb.EINVAL
    assert L.rb_validate(None, None, 1, 1, 1, None, None, None, 1, 1, None, None) == rb.EINVAL
    assert L.rb_greedy_streamed(None, None, 1, 1, 1, 0.0, 1, -1, 0, None) == rb.EINVAL
    assert L.rb_streamed_stats(None, None, None, None) == rb.EINVAL
