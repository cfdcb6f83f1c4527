"""Convolution stacks the throughput measurements run (layer shapes only).

Each layer is (Cin, Cout, H, W, k, stride, pad).  In these measurements the
inputs of every layer are independent fresh encryptions of synthetic
activations of that shape; the chain from one layer to the next through the
x^2 + x protocol is built and tested on its own (the x2x rounds).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    L: int
    B: int
    layers: tuple


def resnet18_cifar():
    """ResNet-18 on 3x32x32: 3x3 stem to 64 channels, four stages of two
    BasicBlocks at 64/128/256/512 channels on 32/16/8/4 pixels; the first 3x3
    conv of stages 2-4 has stride 2 and a 1x1 stride-2 shortcut: 20 convs."""
    layers = [(3, 64, 32, 32, 3, 1, 1)]
    layers += [(64, 64, 32, 32, 3, 1, 1)] * 4
    h, cin = 32, 64
    for width in (128, 256, 512):
        layers.append((cin, width, h, h, 3, 2, 1))
        layers.append((cin, width, h, h, 1, 2, 0))
        h //= 2
        layers += [(width, width, h, h, 3, 1, 1)] * 3
        cin = width
    assert len(layers) == 20
    return tuple(layers)


def resnet50_imagenet():
    """ResNet-50 on 3x224x224: 7x7/2 stem to 64 channels (112x112), then
    (after the pooling layer, not a convolution) bottleneck stages of 3/4/6/3
    blocks at widths 64/128/256/512 (expansion 4) on 56/28/14/7 pixels; stride
    2 on the 3x3 conv of the first block of stages 2-4, 1x1 projection
    shortcuts on every first block: 53 convs."""
    layers = [(3, 64, 224, 224, 7, 2, 3)]
    h, cin = 56, 64
    for si, (width, blocks) in enumerate(((64, 3), (128, 4), (256, 6), (512, 3))):
        for b in range(blocks):
            s = 2 if (b == 0 and si > 0) else 1
            layers.append((cin, width, h, h, 1, 1, 0))
            layers.append((width, width, h, h, 3, s, 1))
            ho = h // s
            layers.append((width, 4 * width, ho, ho, 1, 1, 0))
            if b == 0:
                layers.append((cin, 4 * width, h, h, 1, s, 0))
            cin, h = 4 * width, ho
    assert len(layers) == 53
    return tuple(layers)


WORKLOADS = {
    "single": Workload("single conv 3x3 16->16 on 16x16, B=1, N=4096, L=2", 4096, 2, 1,
                       ((16, 16, 16, 16, 3, 1, 1),)),
    "resnet18": Workload("ResNet-18 CIFAR conv stack (20 convs), B=1, N=8192, L=3", 8192, 3, 1, resnet18_cifar()),
    "resnet18-b64": Workload("ResNet-18 CIFAR conv stack (20 convs), B=64, N=8192, L=3", 8192, 3, 64,
                             resnet18_cifar()),
    "resnet50-b8": Workload("ResNet-50 ImageNet conv stack (53 convs), B=8, N=16384, L=4", 16384, 4, 8,
                            resnet50_imagenet()),
}
