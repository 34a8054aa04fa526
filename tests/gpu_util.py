"""Small helpers shared by the GPU tests: moving numpy arrays to the device and back,
and the score-error measure used against the fp64 oracle."""
import numpy as np
import torch


def dev_u8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def dev_u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).cuda()


def dev_f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host_u16(t):
    return t.cpu().numpy().view(np.uint16)


def host_bits32(t):
    return t.float().cpu().numpy().view(np.uint32)


def rbf_error_scale(x64, sv64, a, b, gamma):
    """sum_i |a_ci| K_i + |b_c| per (row, class): the denominator of the relative score error."""
    d2 = (x64 ** 2).sum(1)[:, None] + (sv64 ** 2).sum(1)[None, :] - 2.0 * x64 @ sv64.T
    K = np.exp(-gamma * np.maximum(d2, 0.0))
    return K @ np.abs(a.astype(np.float64)).T + np.abs(b.astype(np.float64))[None, :]


def rel_score_error(scores, ref, scale):
    return float(np.max(np.abs(scores.astype(np.float64) - ref) / scale))
