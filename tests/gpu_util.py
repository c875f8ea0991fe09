"""Helpers for the GPU parity tests: device placement of synthetic latents."""
import numpy as np
import pytest
import torch

from paper_2509_18815_gb300 import synth


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2509_18815_gb300 import build
    build.build()


def dev_params(params: np.ndarray, bf16: bool = False) -> torch.Tensor:
    if bf16:
        bits = synth.to_bf16_bits(params)
        return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16).contiguous()
    return torch.from_numpy(np.ascontiguousarray(params, np.float32)).cuda()


def oracle_params(params: np.ndarray, bf16: bool = False) -> np.ndarray:
    """The fp32 values the GPU sees (bf16 expands exactly to fp32)."""
    if bf16:
        return synth.bf16_bits_to_f32(synth.to_bf16_bits(params)).reshape(params.shape)
    return np.ascontiguousarray(params, np.float32)


def dev_i32(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def host_u16(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint16)


def host_u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)
