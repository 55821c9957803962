"""Helpers of the GPU tests: device transfer and error measures."""
import numpy as np

import paper_2501_04684_gb300 as ie


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    return torch


def dev(a: np.ndarray):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def empty(shape):
    torch = torch_cuda()
    return torch.zeros(shape, dtype=torch.complex64, device="cuda")


def host(t) -> np.ndarray:
    torch = torch_cuda()
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


def plan_for(p, precs=(ie.IE_PREC_FP32,), max_rhs=1):
    return ie.Plan(ie.problem_from(p, ie.precmask(*precs), max_rhs))


def box_errors(got, ref, nb_targets) -> np.ndarray:
    """Relative L2 error of every target box (rows concatenated in target order, nb_t
    rows each), over all right-hand sides: a fault confined to a few boxes or to one
    displacement class shows here even when the vector-wide error stays small."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    off = np.concatenate([[0], np.cumsum(np.asarray(nb_targets))])
    return np.array([np.linalg.norm(got[..., off[i]:off[i + 1]] - ref[..., off[i]:off[i + 1]]) /
                     np.linalg.norm(ref[..., off[i]:off[i + 1]]) for i in range(len(off) - 1)])
