"""The C-ABI library builds and exports every entry point its headers declare
(no GPU needed: symbols are resolved, nothing is called)."""

import ctypes
import os
import re

from paper_2603_25260_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in ("lpc.h", "lpc_ops.h", "lpc_train.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            if m.group(1) not in ("if", "defined"):
                names.add(m.group(1))
    return names


def test_headers_declare_the_boundary():
    names = _declared()
    for want in ("codec_create", "codec_destroy", "codec_last_error", "encode_frame",
                 "decode_frame", "probs_level", "encode_batch", "decode_batch",
                 "lpc_build_levels", "lpc_kernel_map", "lpc_conv333", "lpc_down_s2",
                 "lpc_up_prune", "lpc_softmax_cdf", "lpc_kernel_map_noalloc",
                 "lpc_kernel_map_child",
                 "lpc_t_conv_fwd", "lpc_t_conv_bwd", "lpc_t_up_fwd", "lpc_t_up_bwd",
                 "lpc_t_down_fwd", "lpc_t_down_bwd", "lpc_t_embed_fwd", "lpc_t_embed_bwd",
                 "lpc_t_prelu_fwd", "lpc_t_prelu_bwd", "lpc_t_fq_fwd", "lpc_t_fq_bwd", "lpc_t_fq_w",
                 "lpc_t_levels", "codec_tuning", "lpc_conv333_variant", "lpc_up_prune_variant",
                 "codec_set_tuning"):
        assert want in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
