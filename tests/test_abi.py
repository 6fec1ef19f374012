"""The C-ABI library builds, loads on a machine without a GPU, exports every
entry point include/alto.h declares, and its host-only entry points agree
with the oracle (no compute call needs a GPU here)."""
import os
import re

import numpy as np
import pytest

import oracle

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "alto.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:alto_status|const\s+char\s*\*)\s*(alto_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("alto_create", "alto_mttkrp", "alto_cpals", "alto_destroy", "alto_export", "alto_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(alto_lib):
    for name in declared():
        assert hasattr(alto_lib, name), name


def _oracle_masks(dims):
    nbits, pos, B = oracle.bit_map(dims)
    masks = []
    for n in range(len(dims)):
        lo = hi = 0
        for l in range(nbits[n]):
            p = int(pos[n][l])
            if p < 64:
                lo |= 1 << p
            else:
                hi |= 1 << (p - 64)
        masks.append((lo, hi))
    return list(nbits), masks, B


@pytest.mark.parametrize("dims", [(4, 8, 2), (64, 128, 256), (4_000_000, 4_000_000, 30_000),
                                  (12_000, 60_000, 5_000_000, 100), (1 << 20,) * 3 + (1 << 16,) * 2,
                                  (1, 1, 1), (2 ** 32, 5), (3, 3, 3, 3, 3, 3, 3, 3), (7,)])
def test_layout_matches_oracle(alto_lib, dims):
    from paper_2102_10245_gb300 import layout_for_dims
    bits, masks, kw, B = layout_for_dims(dims)
    obits, omasks, oB = _oracle_masks(dims)
    assert bits == obits and masks == omasks and B == oB
    assert kw == (1 if B <= 64 else 2)


def test_key_width_override(alto_lib):
    from paper_2102_10245_gb300 import layout_for_dims, AltoError
    assert layout_for_dims((64, 128, 256), key_bits=128)[2] == 2
    assert layout_for_dims((64, 128, 256), key_bits=64)[2] == 1
    with pytest.raises(AltoError) as e:
        layout_for_dims((1 << 20,) * 3 + (1 << 16,) * 2, key_bits=64)
    assert e.value.status == 5          # ALTO_EOVERFLOW


@pytest.mark.parametrize("dims", [(), (0, 4), (2 ** 32 + 1, 2), tuple([2] * 9)])
def test_layout_rejects_bad_dims(alto_lib, dims):
    from paper_2102_10245_gb300 import layout_for_dims, AltoError
    with pytest.raises(AltoError) as e:
        layout_for_dims(dims)
    assert e.value.status == 1          # ALTO_EINVAL


def test_layout_rejects_more_than_128_bits(alto_lib):
    from paper_2102_10245_gb300 import layout_for_dims, AltoError
    with pytest.raises(AltoError) as e:
        layout_for_dims((2 ** 32,) * 5)   # 160 bits
    assert e.value.status == 5


@pytest.mark.parametrize("dims", [(4, 8, 2), (4_000_000, 4_000_000, 30_000), (12_000, 60_000, 5_000_000, 100),
                                  (1 << 20,) * 3 + (1 << 16,) * 2, (2 ** 32, 3, 1), (5, 9, 17, 33, 65, 129, 3, 2)])
def test_host_decode_matches_oracle(alto_lib, dims):
    """The precomputed compress masks the kernels use de-linearize exactly
    like the oracle's bit-by-bit decode."""
    from paper_2102_10245_gb300 import decode_host, layout_for_dims
    rng = np.random.default_rng(0)
    coords = np.stack([rng.integers(0, d, 2000, dtype=np.int64) for d in dims], 1)
    coords[0] = [d - 1 for d in dims]
    coords[1] = 0
    keys = oracle.encode(dims, [coords[:, n] for n in range(len(dims))])
    kw = layout_for_dims(dims)[2]
    got = decode_host(dims, keys[:, :kw])
    assert (got.astype(np.int64) == coords).all()


def test_argument_errors_need_no_gpu(alto_lib):
    """Entry points reject bad arguments on the host, before any CUDA call:
    a NULL tensor handle, an unknown Gram engine, a bad Gram shape, and the
    tensor-core engine asked for FP32 factors or a rank it has no kernel for."""
    import ctypes
    L = alto_lib
    modes = (ctypes.c_int * 1)(0)
    assert L.alto_transpose(None, 1, modes, None, None, None, 8, None, None) == 1
    assert L.alto_set_gram_engine(None, 0) == 1
    dummy = ctypes.c_void_p(16)
    G = ctypes.c_void_p(32)
    assert L.alto_gram(dummy, 10, 32, 2, 7, G, None) == 1          # engine out of range
    assert L.alto_gram(dummy, 10, 65, 2, 0, G, None) == 1          # R above 64
    assert L.alto_gram(dummy, -1, 32, 2, 0, G, None) == 1          # negative length
    assert L.alto_gram(dummy, 10, 32, 2, 0, None, None) == 1       # NULL output
    assert L.alto_gram(None, 10, 32, 2, 0, G, None) == 1           # NULL factor
    assert L.alto_gram(dummy, 10, 32, 1, 2, G, None) == 1          # tensor cores with FP32 factors
    assert L.alto_gram(dummy, 10, 24, 2, 2, G, None) == 1          # tensor cores at R = 24
