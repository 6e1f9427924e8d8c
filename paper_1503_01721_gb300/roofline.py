"""Algorithmic byte counts and measured peaks used to report roofline fractions.

Byte model of one sparse product over a CSR matrix (the format's own bytes,
no padding): every stored nonzero moves its value and its 4-byte column index
once; the row pointers (8 bytes each), the dense input and the dense output
move once.  Section 3.2, Table 2 of the paper fixes 8 bytes per nonzero for a
float32 CSR and 12 bytes per nonzero for COO.
"""
from __future__ import annotations

import json
import os

VAL_BYTES = {"f32": 4, "bf16": 2, "fp8": 1}
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy bandwidth is the roofline denominator)
IDX_BYTES = 4
PTR_BYTES = 8


def csr_bytes_per_nnz(dtype: str = "f32") -> int:
    return VAL_BYTES[dtype] + IDX_BYTES


def coo_bytes_per_nnz() -> int:
    return 4 + 2 * IDX_BYTES


def spmv_bytes(nnz: int, n_rows: int, n_in: int, n_out: int, dtype: str = "f32", n_scales: int = 0) -> int:
    """Algorithmic bytes of y = M x for a CSR matrix M (n_rows rows, nnz nonzeros)."""
    return (nnz * csr_bytes_per_nnz(dtype) + PTR_BYTES * (n_rows + 1)
            + 4 * n_in + 4 * n_out + 4 * n_scales)


def spmv_bytes_index16(nnz: int, n_chunks: int, n_rows: int, n_in: int, n_out: int, dtype: str = "f32",
                       n_scales: int = 0) -> int:
    """Algorithmic bytes of y = M x reading the 16-bit column index: 2 bytes per
    nonzero, a 4-byte base per 128-entry chunk and an 8-byte chunk pointer per row
    replace the 4-byte index."""
    return (nnz * (VAL_BYTES[dtype] + 2) + 4 * n_chunks + 2 * PTR_BYTES * (n_rows + 1)
            + 4 * n_in + 4 * n_out + 4 * n_scales)


def measured_peaks(path: str | None = None) -> dict:
    """Peaks measured on this GPU model (copy bandwidth, bf16 GEMM), if recorded."""
    if path is None:
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}
