"""Convenience wrapper: a pattern table plus PyTorch-owned device buffers.

Every step of a search runs in ``librk.so``; this class only allocates the
output, result header and workspace tensors and reads the match count back.
"""

from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import rk


class Matcher:
    def __init__(self, patterns: Sequence[bytes], **opts):
        self.patterns = [bytes(p) for p in patterns]
        self.table = rk.rk_build(self.patterns, **opts)
        self.info = rk.rk_table_info(self.table)

    def close(self) -> None:
        if self.table:
            rk.rk_destroy(self.table)
            self.table = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def search(self, text: torch.Tensor, capacity: Optional[int] = None,
               stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """Sorted match keys (id << 40 | x) of a uint8 CUDA tensor.  The
        workspace holds the sort's scratch and the candidate list, so the
        scan verifies its survivors in a second kernel when the table allows."""
        assert text.is_cuda and text.dtype == torch.uint8 and text.is_contiguous()
        n = text.numel()
        cap = capacity if capacity is not None else max(1024, n // 256)
        st = stream or torch.cuda.current_stream(text.device)
        scan_b = rk.rk_scan_workspace_bytes(self.table, n)
        while True:
            keys = torch.empty(max(cap, 1), dtype=torch.int64, device=text.device)
            info = torch.zeros(2, dtype=torch.int64, device=text.device)
            wsb = rk.rk_workspace_bytes(self.table, cap) + scan_b
            ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=text.device)
            rk.rk_search_device(self.table, text if n else 0, n, keys, cap, info, ws, wsb, st)
            st.synchronize()
            count, status = (int(v) for v in info.cpu().tolist())
            if status != rk.RK_OK:
                raise rk.RkError(status, "search")
            if count <= cap:
                return keys[:count]
            cap = count
