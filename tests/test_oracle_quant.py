"""Pins for the oracle's BF16 / FP8 E4M3 encoders: format-definition values and library casts."""
import numpy as np
import torch

from oracle import quant


def test_bf16_known_codes_and_ties():
    vals = np.array([1.0, -2.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.0e38, 0.0, -0.0], dtype=np.float32)
    # 1+2^-8 is halfway between 1 and 1+2^-7: ties to even -> 1.0 ; 1+3*2^-8 -> 1+2^-6
    assert quant.bf16_bits(vals).tolist() == [0x3F80, 0xC000, 0x3F80, 0x3F82, 0x7F62, 0x0000, 0x8000]


def test_bf16_matches_torch_cast():
    rng = np.random.default_rng(0)
    x = (rng.normal(0, 1, 200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    # exact ties too: values with the low 16 bits equal to 0x8000
    ties = (rng.integers(0, 1 << 31, 5000, dtype=np.int64).astype(np.uint32) & 0xFFFF0000 | 0x8000).view(np.float32)
    x = np.concatenate([x, ties[np.isfinite(ties)]])
    want = torch.tensor(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert (quant.bf16_bits(x) == want).all()


def test_e4m3_known_codes():
    vals = [448.0, 1.0, 2.0 ** -9, 1.0625, 1.1875, 500.0, -1.0, 0.0, 2.0 ** -6, 2.0 ** -10, 3 * 2.0 ** -10, 464.0]
    # 1.0625 is halfway 1.0 (0x38) / 1.125 (0x39): even -> 0x38 ; 1.1875 halfway 0x39/0x3A -> 0x3A
    # 2^-10 halfway 0 / 2^-9: even -> 0 ; 3*2^-10 halfway 2^-9 / 2^-8: even (m=2) -> 0x02
    # 464 = 448 + half an ulp: saturates to 448
    want = [0x7E, 0x38, 0x01, 0x38, 0x3A, 0x7E, 0xB8, 0x00, 0x08, 0x00, 0x02, 0x7E]
    assert quant.e4m3_bits(vals).tolist() == want


def test_e4m3_all_codes_round_trip():
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], dtype=np.uint8)
    vals = quant.e4m3_value(codes)
    back = quant.e4m3_bits(vals)
    # +0 and -0 both decode to a zero; everything else is a bijection
    assert (back == codes).all()


def test_e4m3_matches_torch_cast_in_range():
    rng = np.random.default_rng(1)
    x = (rng.normal(0, 1, 100000) * np.exp(rng.uniform(-9, 6, 100000))).astype(np.float32)
    x = x[np.abs(x) <= 448.0]
    mids = (quant.e4m3_value(np.arange(0, 0x7E)) + quant.e4m3_value(np.arange(1, 0x7F))) / 2
    x = np.concatenate([x, mids.astype(np.float32), -mids.astype(np.float32)])
    want = torch.tensor(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert (quant.e4m3_bits(x) == want).all()
