"""Pins for the oracle's storage rounding (bfloat16 and binary16, round to
nearest even): compared with torch's and numpy's own conversions on every
exponent, around every rounding boundary, on a random sample of bit patterns
and (marked slow) on all 2^32 of them.  NaNs are compared by class only."""
import numpy as np
import pytest
import torch


def patterns():
    rng = np.random.default_rng(1234)
    rand = rng.integers(0, 2 ** 32, size=1 << 21, dtype=np.uint64).astype(np.uint32)
    # every sign and exponent, with low halves around the bf16 and f16 boundaries
    hi = np.arange(0, 1 << 9, dtype=np.uint32) << np.uint32(23)
    lows = [0, 1, 0x0FFF, 0x1000, 0x1001, 0x1FFF, 0x2000, 0x3000, 0x7FFF, 0x8000, 0x8001,
            0xFFFF, 0x10000, 0x18000, 0x7FFFFF, 0x400000, 0x3FFFFF, 0x401000, 0x7FE000]
    # binary16 subnormal boundaries: the discarded-bit count goes up to 24
    lows += [(1 << s) - 1 for s in range(1, 24)] + [1 << s for s in range(0, 23)]
    lows += [(1 << s) | (1 << (s - 1)) for s in range(1, 23)]
    edge = (hi[:, None] | np.array(lows, dtype=np.uint32)[None, :]).ravel()
    return np.concatenate([rand, edge]).view(np.float32)


def test_bf16_matches_torch(orc):
    x = patterns()
    ours = orc.f32_to_bf16_array(x)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    nan = np.isnan(x)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert np.all((ours[nan] & 0x7F80) == 0x7F80) and np.all(ours[nan] & 0x7F)


def test_f16_matches_numpy(orc):
    x = patterns()
    ours = orc.f32_to_f16_array(x)
    ref = x.astype(np.float16).view(np.uint16)
    nan = np.isnan(x)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert np.all((ours[nan] & 0x7C00) == 0x7C00) and np.all(ours[nan] & 0x3FF)


def test_f16_decode_matches_numpy(orc):
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    ours = orc.f16_bits_to_f32_array(bits)
    ref = bits.view(np.float16).astype(np.float32)
    nan = np.isnan(ref)
    assert np.array_equal(ours[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    assert np.all(np.isnan(ours[nan]))


def test_round_storage_roundtrip(orc):
    x = np.array([1.0, 1.00390625, 1.005859375, 3.0e-8, 65504.0, 65520.0], dtype=np.float32)
    b = orc.round_storage(x, "bf16")
    assert np.array_equal(b, torch.from_numpy(x).to(torch.bfloat16).float().numpy())
    h = orc.round_storage(x, "f16")
    assert np.array_equal(h, x.astype(np.float16).astype(np.float32))
    assert np.array_equal(orc.round_storage(x, "f32"), x)


@pytest.mark.slow
def test_bf16_and_f16_over_every_binary32_pattern(orc):
    # All 2^32 bit patterns, in chunks: the oracle's bit-level rounding to
    # nearest even against torch's bfloat16 and binary16 conversions (their
    # own implementations of the same rule); NaNs by class.
    chunk = 1 << 25
    base = np.arange(chunk, dtype=np.uint32)
    for c in range((1 << 32) // chunk):
        x = (base + np.uint32(c * chunk)).view(np.float32)
        ob = orc.f32_to_bf16_array(x)
        tb = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        oh = orc.f32_to_f16_array(x)
        nh = torch.from_numpy(x).to(torch.float16).view(torch.int16).numpy().view(np.uint16)
        for ours, ref, exp_mask, man_mask in ((ob, tb, 0x7F80, 0x7F), (oh, nh, 0x7C00, 0x3FF)):
            diff = ours != ref
            if diff.any():
                assert np.all(np.isnan(x[diff])), f"chunk {c}: non-NaN input rounded differently"
                bad = ours[diff]
                assert np.all((bad & exp_mask) == exp_mask) and np.all(bad & man_mask)
