"""Transfer arenas for a step's inputs and outputs.

A one-call step reads many buffers (the occupancy prior or coordinates, a depth
raster and a mask per view, the points) and writes a few (the seg bitfield, the
point labels).  Copied one by one, the small copies each pay the transfer's
fixed cost; here the buffers of one direction live in one pinned host arena and
one device arena, each buffer a view at a 256-byte aligned offset of both, so
that a step's host-to-device traffic is one copy and its device-to-host
traffic another.  A producer writes a step's inputs straight into the host
views (``host[name]``) and the kernels read the device views
(``device[name]``).  Plain PyTorch copies: no arithmetic of the method here.
"""
from __future__ import annotations

from typing import Dict, Iterable, Tuple

import torch

_ALIGN = 256


class Arena:
    """Named buffers laid out back to back (256-byte aligned) in one pinned
    host tensor and one device tensor of the same size."""

    def __init__(self, specs: Iterable[Tuple[str, Tuple[int, ...], torch.dtype]], device):
        self.offsets: Dict[str, Tuple[int, int]] = {}
        off = 0
        layout = []
        for name, shape, dtype in specs:
            if name in self.offsets:
                raise ValueError(f"duplicate buffer name {name!r}")
            n = 1
            for d in shape:
                n *= int(d)
            nbytes = n * torch.empty((), dtype=dtype).element_size()
            off = (off + _ALIGN - 1) // _ALIGN * _ALIGN
            self.offsets[name] = (off, nbytes)
            layout.append((name, tuple(int(d) for d in shape), dtype, off, nbytes))
            off += nbytes
        self.nbytes = max(off, 1)
        self.host_bytes = torch.empty(self.nbytes, dtype=torch.uint8).pin_memory()
        self.device_bytes = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.host: Dict[str, torch.Tensor] = {}
        self.device: Dict[str, torch.Tensor] = {}
        for name, shape, dtype, o, nb in layout:
            self.host[name] = self.host_bytes[o:o + nb].view(dtype).view(shape)
            self.device[name] = self.device_bytes[o:o + nb].view(dtype).view(shape)

    def payload_bytes(self) -> int:
        """Bytes of the buffers themselves (without the alignment gaps)."""
        return sum(nb for _, nb in self.offsets.values())

    def upload(self, stream: torch.cuda.Stream | None = None) -> None:
        """All buffers host -> device in one asynchronous copy on ``stream``."""
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            self.device_bytes.copy_(self.host_bytes, non_blocking=True)

    def download(self, stream: torch.cuda.Stream | None = None) -> None:
        """All buffers device -> host in one asynchronous copy on ``stream``."""
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            self.host_bytes.copy_(self.device_bytes, non_blocking=True)
