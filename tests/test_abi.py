"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point that include/cachedconv.h declares, and its
planning pass reproduces the oracle's section 3 analysis (Eq. 2 / Eq. 3
delays, kept frames) without touching device memory."""
import os
import re

import numpy as np
import pytest

from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "cachedconv.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(cclib):
    names = _declared()
    assert "cc_model_create" in names and "cc_stream_process" in names
    for name in names:
        assert hasattr(cclib, name), name
    assert set(api.EXPORTED) <= set(names)


def _plan(nodes):
    return api.Model(nodes, {}, max_streams=0)


def _autoencoder():
    return W.chain(W.rave_encoder(), W.rave_decoder())


@pytest.mark.parametrize("builder", [W.tiny_stack, W.rave_decoder, W.rave_encoder, _autoencoder])
def test_plan_matches_oracle_analysis(cclib, builder):
    nodes = builder()
    info = M.analyze(nodes)
    keep = M.cache_frames(nodes, info)
    m = _plan(nodes)
    assert m.total_delay == info["delay"]
    io = m.io
    assert io["in_per_step"] == info["in_per_step"]
    for i, nd in enumerate(nodes):
        ni = m.node_info(i)
        assert ni["delay"] == info["D"][i], (i, nd["name"])
        assert ni["extra_delay"] == info["Da"][i]
        assert ni["align"][:len(info["A"][i])] == info["A"][i]
        assert ni["kept"] == keep[i]
        assert ni["frames_per_step"] == info["rate"][i] * info["in_per_step"]
    state, slot = m.state_bytes
    assert state == 4 * M.cache_elements(nodes, info)
    m.close()


def test_audio_to_audio_delay_composes(cclib):
    """Delays compose through a chain (section 3.1): the encoder's 3-frame
    latent delay reaches the output as 3 x 2048 samples on top of the
    decoder's own 12424."""
    m = _plan(_autoencoder())
    assert m.total_delay == 3 * 2048 + 12424
    assert m.io == dict(in_channels=1, out_channels=1, in_per_step=2048, out_per_step=2048)
    m.close()


def test_decoder_plan_numbers(cclib):
    m = _plan(W.rave_decoder())
    assert m.total_delay == 12424
    assert m.io == dict(in_channels=128, out_channels=1, in_per_step=1, out_per_step=2048)
    assert m.state_bytes[0] == 27648 * 4


@pytest.mark.parametrize("mutate,msg", [
    (lambda n: n.__setitem__(1, dict(n[1], inputs=[5])), "earlier node"),
    (lambda n: n.__setitem__(1, dict(n[1], c_in=7)), "c_in"),
    (lambda n: n.__setitem__(1, dict(n[1], pad_left=0, pad_right=0)), "looks ahead"),
    (lambda n: n.__setitem__(0, dict(n[0], op="conv", inputs=[])), "input"),
])
def test_bad_graphs_are_rejected(cclib, mutate, msg):
    nodes = W.tiny_stack()
    mutate(nodes)
    with pytest.raises(api.CCError) as e:
        _plan(nodes)
    assert e.value.status == -2 and msg in str(e.value)


def test_bad_convt_rejected(cclib):
    nodes = [W.input_node(4), W._node("convt", [0], 4, 4, k=6, stride=4, crop=1)]
    with pytest.raises(api.CCError) as e:
        _plan(nodes)
    assert "multiple of its stride" in str(e.value)


def test_merge_rate_mismatch_rejected(cclib):
    nodes = [W.input_node(2), W._node("conv", [0], 2, 2, k=3, stride=2, pad_left=1, pad_right=1),
             W._node("add", [0, 1], 2, 2, bias=False)]
    with pytest.raises(api.CCError) as e:
        _plan(nodes)
    assert "rates" in str(e.value)


def test_host_pqmf_design_matches_oracle(cclib):
    for bands, taps, beta in [(16, 64, 5.0), (16, 128, 8.0), (4, 64, 9.0)]:
        h, g, wc = api.pqmf_design(bands, taps, beta)
        h2, g2, _, wc2 = pqmf.design(bands, taps, beta)
        np.testing.assert_allclose(h, h2, atol=1e-13)
        np.testing.assert_allclose(g, g2, atol=1e-13)
        assert abs(wc - wc2) < 1e-12


def test_host_pqmf_layer_weights_match_oracle(cclib):
    """The PQMF layers' trained-layout weights come from the library: analysis
    conv g_b, synthesis convT bands * g_b (float32 of the same design)."""
    a, s = api.pqmf_layer_weights(16, 64, 5.0)
    _, g, _, _ = pqmf.design(16, 64, 5.0)
    assert a.shape == s.shape == (16, 1, 64) and a.dtype == s.dtype == np.float32
    np.testing.assert_allclose(a, pqmf.analysis_weights(g), rtol=0, atol=1e-7)
    np.testing.assert_allclose(s, pqmf.synthesis_weights(g), rtol=0, atol=16e-7)


def test_missing_library_fails_loudly():
    """No CPU fallback: with the library absent, the first call raises."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = f"""
import sys
sys.path.insert(0, {root!r})
from paper_2204_07064_gb300 import build, api, workloads as W
build.LIB = "/nonexistent/libcachedconv.so"
try:
    api.Model(W.tiny_stack(), {{}}, max_streams=0)
except RuntimeError as e:
    assert "not built" in str(e), e
    print("raised")
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "raised"


def test_product_package_never_imports_the_oracle():
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = f"""
import sys
sys.path.insert(0, {root!r})
import paper_2204_07064_gb300
from paper_2204_07064_gb300 import api, autograd, workloads, build
assert not any(m == "oracle" or m.startswith("oracle.") for m in sys.modules), sorted(sys.modules)
print("clean")
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "clean"
    pkg = os.path.join(root, "paper_2204_07064_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), f


def test_binding_argument_counts_match_the_header():
    """Every ctypes signature of the Python binding has as many arguments as the
    C declaration (a missing or extra argument would shift the others)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = {}
    for m in re.finditer(r"\b(cc_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        params = m.group(2).strip()
        decls[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    for name, argtypes in api._SIGNATURES.items():
        assert name in decls, name
        assert len(argtypes) == decls[name], (name, len(argtypes), decls[name])


def test_binding_argument_types_match_the_header():
    """Scalar widths and pointer-ness of every argument agree with the header
    (an int32 passed for an int64 would leave the upper half undefined)."""
    import ctypes as C

    scalar = {"int32_t": C.c_int32, "cc_status": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64,
              "size_t": C.c_size_t,
              "double": C.c_double}
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for m in re.finditer(r"\b(cc_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        name, params = m.group(1), m.group(2).strip()
        if name not in api._SIGNATURES or params in ("", "void"):
            continue
        for i, (decl, t) in enumerate(zip(params.split(","), api._SIGNATURES[name])):
            decl = " ".join(decl.split())
            if "*" in decl:
                is_ptr = t is C.c_void_p or t is C.c_char_p or (isinstance(t, type) and issubclass(t, C._Pointer))
                assert is_ptr, (name, i, decl, t)
            else:
                ctype = decl.replace("const ", "").split()[0]
                assert ctype in scalar, (name, i, decl)
                assert t is scalar[ctype], (name, i, decl, t)


C_PROGRAM = r"""
#include <stdio.h>
#include "cachedconv.h"
int main(void) {
  cc_node_desc nodes[2] = {0};
  nodes[0].op = CC_OP_INPUT; nodes[0].c_in = 4; nodes[0].c_out = 4;
  nodes[1].op = CC_OP_CONV; nodes[1].n_inputs = 1; nodes[1].inputs[0] = 0;
  nodes[1].c_in = 4; nodes[1].c_out = 4; nodes[1].kernel = 3; nodes[1].stride = 1;
  nodes[1].dilation = 1; nodes[1].pad_left = 1; nodes[1].pad_right = 1; nodes[1].has_bias = 1;
  cc_model_config cfg = {CC_F32, 0, 1, 1, 0, 0, 0};
  cc_model* m = NULL;
  cc_status s = cc_model_create(nodes, 2, NULL, NULL, &cfg, &m);
  if (s != CC_OK) { printf("create: %s %s\n", cc_status_str(s), cc_last_error()); return 1; }
  int64_t d = -1;
  s = cc_model_total_delay(m, &d);
  printf("%d %lld\n", (int)s, (long long)d);
  cc_model_destroy(m);
  return 0;
}
"""


def test_c_program_uses_the_abi(cclib):
    """The header is plain C (C99, no warnings) and a C program links against
    the library: a plan-only model (no GPU needed) of one k=3 conv with pads
    1/1 reports the one-frame delay of the causal reconfiguration (section 3)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(api.library_path())
    exe = os.path.join(libdir, "abi_c_check")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(root, "include"), "-x", "c", "-", "-L", libdir, "-lcachedconv",
                        "-Wl,-rpath," + libdir, "-o", exe], input=C_PROGRAM, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.split() == ["0", "1"]
