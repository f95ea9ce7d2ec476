"""Surrogate tensor-core kernels at the production shape against oracle/cnn.py.

The network of the bench works on 256 x 256 lattices, where a row holds two
128-pixel tiles (the halo pixels at the seam between them are interior pixels,
not wrapped ones) and every CTA of the ring convolutions walks a strip of
several rows, so its shared-memory ring of input rows turns over many times.
These tests run that shape, a ragged one (odd H = 131, where strips end and
restart at rows that are not multiples of the 8-slot ring, W = 384: three tiles
per row) and the smallest lattice (H = 3, every halo row wrapped), on both
tensor paths (tcgen05 and mma.sync), and compare with the FP64 oracle:

1. Per operation, on the GPU's own bf16 inputs (only that operation's rounding
   differs): every forward convolution (4 -> 64, 4 x 64 -> 64, 64 -> 4), every
   backward-data convolution with its ReLU mask (the tcgen05 path rounds the
   output layer's FP32 upstream gradient to bf16 first, as the network keeps
   every other gradient), every weight and bias gradient.
2. Along the oracle's own chain: a forward and backward pass computed entirely
   by the oracle from the same bf16 input, bf16 weights and upstream gradient,
   with every stored activation and gradient rounded to bf16 as the network
   stores them.  The GPU's activations, backward-data gradients and weight
   gradients are compared with the oracle's, so that an error in one layer
   cannot hide behind the next layer being fed the GPU's own output.

Tolerances.  (1) is the final bf16 rounding: 2^-8 relative per element plus
1e-5 of the tensor's maximum; FP32 results (the 64 -> 4 output and the weight
gradients, FP32 accumulation over up to 2 x 10^5 pixels) 1e-5 and 1e-3 of the
maximum.  (2): GPU (FP32 accumulation) and oracle (FP64) round a value to a
different bf16 neighbour when it lies within their accumulation difference of
a rounding midpoint; such one-unit flips (2^-8 relative) then feed the next
layer.  The forward pass is continuous in its inputs, so the activations and
the output stay within 2^-6 of the tensor's maximum element by element
(measured <= 5.1e-3).  The backward pass is not: the ReLU mask is a decision,
and where a pre-activation lies within that noise of zero the two sides decide
differently and the gradient there is either passed whole or dropped.  Such
flips are rare (measured <= 3.3e-5 of the entries of a layer, bound 1e-4), but
each carries a full-size gradient, so the backward-data gradients are compared
in relative L2 norm (measured <= 1.1e-2, bound 3e-2) and the weight and bias
gradients, sums over the lattice, against 3e-2 of their maximum (measured
<= 1.3e-2); a wrong tap, operand or mask would be off by O(1).
"""
import numpy as np
import pytest

import oracle as O  # noqa: F401  (builds the oracle library on first use)
from oracle import cnn as N
from paper_1402_5487_gb300 import build, plbm
from paper_1402_5487_gb300 import surrogate as SG

pytestmark = pytest.mark.gpu

CIN = [4, 64, 64, 64, 64, 64]
COUT = [64, 64, 64, 64, 64, 4]
SHAPES = [(2, 256, 256), (3, 131, 384), (1, 3, 128)]


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as FP64."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split(p):
    out, k = [], 0
    for ci, co in zip(CIN, COUT):
        n = 9 * ci * co
        W = p[k:k + n].reshape(3, 3, ci, co).astype(np.float64)
        k += n
        b = p[k:k + co].astype(np.float64)
        k += co
        out.append((W, b))
    return out


def close_bf16(gpu, ref):
    scale = np.max(np.abs(ref))
    return bool(np.all(np.abs(gpu - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * scale))


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def oracle_chain(x, params, dout):
    """Forward and backward pass of the network by the oracle, with the stored
    activations (after ReLU) and backward-data gradients rounded to bf16 and the
    weights taken in bf16, as the network keeps them.  Returns the layer inputs
    A[0..5], the FP32-level output, the upstream gradients of each layer's
    convolution output ups[0..5] and the weight and bias gradients."""
    Wb = [(bf16(W), b) for W, b in params]
    A = [x]
    for l in range(5):
        A.append(bf16(N.relu(N.conv3x3(A[l], Wb[l][0], Wb[l][1]))))
    out = N.conv3x3(A[5], Wb[5][0], Wb[5][1])
    ups = [None] * 6
    ups[5] = dout
    for l in range(5, 0, -1):
        ups[l - 1] = bf16(N.conv3x3_grad_input(ups[l], Wb[l][0]) * (A[l] > 0))
    grads = [N.conv3x3_grad_weight(A[l], ups[l]) for l in range(6)]
    return A, out, ups, grads


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    plbm.lib()


@pytest.fixture(scope="module", params=[(p, s) for p in ("tcgen05", "mma_sync") for s in SHAPES],
                ids=lambda ps: "%s-%dx%dx%d" % ((ps[0],) + ps[1]))
def gpu_pass(request):
    import torch
    path, (B, H, W) = request.param
    net = SG.Surrogate(B, H=H, W=W, seed=7)
    net.set_tensor_path(path == "tcgen05")
    g = torch.Generator().manual_seed(3 + H)
    x = torch.randn((B, H, W, 4), generator=g).to(torch.bfloat16).cuda()
    dout = (0.01 * torch.randn((B, H, W, 4), generator=g)).cuda()
    torch.cuda.synchronize()
    out = net.forward(x, B).cpu().numpy().astype(np.float64)
    A = [x.float().cpu().numpy().astype(np.float64)]
    A += [net.tensor(0, l, B).float().cpu().numpy().astype(np.float64) for l in range(1, 6)]
    grads = split(net.backward(x, dout, B))
    dZ = [net.tensor(1, l, B).float().cpu().numpy().astype(np.float64) for l in range(1, 6)]
    p, _ = net.params()
    assert net.check() == plbm.PLBM_OK
    net.close()
    yield dict(A=A, out=out, dZ=dZ, dout=dout.cpu().numpy().astype(np.float64), params=split(p), grads=grads,
               tc=path == "tcgen05")


def test_each_forward_convolution_on_the_gpu_inputs(gpu_pass):
    A, params = gpu_pass["A"], gpu_pass["params"]
    for l in range(6):
        W, b = params[l]
        ref = N.conv3x3(A[l], bf16(W), b)
        if l < 5:
            assert close_bf16(A[l + 1], N.relu(ref)), l
        else:
            assert max_rel(gpu_pass["out"], ref) < 1e-5


def test_each_backward_data_convolution_on_the_gpu_inputs(gpu_pass):
    # the tcgen05 path takes the output layer's upstream gradient in bf16 (as
    # every other layer's), the mma.sync path in FP32
    A, dZ, params = gpu_pass["A"], gpu_pass["dZ"], gpu_pass["params"]
    dout = gpu_pass["dout"]
    ups = dZ + [bf16(dout) if gpu_pass["tc"] else dout]
    for l in range(5, 0, -1):
        ref = N.conv3x3_grad_input(ups[l], bf16(params[l][0])) * (A[l] > 0)
        assert close_bf16(dZ[l - 1], ref), l


def test_each_weight_gradient_on_the_gpu_inputs(gpu_pass):
    A, dZ, grads = gpu_pass["A"], gpu_pass["dZ"], gpu_pass["grads"]
    ups = dZ + [gpu_pass["dout"]]
    for l in range(6):
        dW, db = N.conv3x3_grad_weight(A[l], ups[l])
        assert max_rel(grads[l][0], dW) < 1e-3, l
        assert max_rel(grads[l][1], db) < 1e-3, l


def l2_rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_whole_pass_along_the_oracle_chain(gpu_pass):
    A, dZ, grads = gpu_pass["A"], gpu_pass["dZ"], gpu_pass["grads"]
    oA, oout, oups, ograds = oracle_chain(A[0], gpu_pass["params"], gpu_pass["dout"])
    for l in range(1, 6):
        assert max_rel(A[l], oA[l]) <= 2.0 ** -6, ("activation", l, max_rel(A[l], oA[l]))
        flips = np.count_nonzero((A[l] > 0) != (oA[l] > 0))
        assert flips <= 1e-4 * A[l].size, ("ReLU decisions", l, flips)
    assert max_rel(gpu_pass["out"], oout) <= 2.0 ** -6, ("output", max_rel(gpu_pass["out"], oout))
    for l in range(5):
        assert l2_rel(dZ[l], oups[l]) <= 3e-2, ("dZ", l, l2_rel(dZ[l], oups[l]))
    for l in range(6):
        assert max_rel(grads[l][0], ograds[l][0]) <= 3e-2, ("dW", l, max_rel(grads[l][0], ograds[l][0]))
        assert max_rel(grads[l][1], ograds[l][1]) <= 3e-2, ("db", l, max_rel(grads[l][1], ograds[l][1]))
