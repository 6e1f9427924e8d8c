"""The byte model used for the GB/s metric reproduces the DDC sizes that
Table 2 (Section 3.2) prints for COO and CSR."""
import os

from paper_1503_01721_gb300 import roofline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_ddc_bytes.txt")


def test_table2_sizes():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for nnz, coo, csr in rows:
        nnz = int(nnz)
        assert round(nnz * roofline.coo_bytes_per_nnz() / 2 ** 30, 2) == float(coo)
        assert round(nnz * roofline.csr_bytes_per_nnz("f32") / 2 ** 30, 2) == float(csr)
        # the paper's "CSR is about 2/3 of COO" (Section 2.2.2)
        assert abs(roofline.csr_bytes_per_nnz("f32") / roofline.coo_bytes_per_nnz() - 2 / 3) < 1e-12


def test_spmv_bytes_counts_each_array_once():
    assert roofline.spmv_bytes(10, 3, 5, 3) == 10 * 8 + 8 * 4 + 4 * 5 + 4 * 3
    assert roofline.spmv_bytes(10, 3, 5, 3, "fp8", n_scales=5) == 10 * 5 + 8 * 4 + 20 + 12 + 20
