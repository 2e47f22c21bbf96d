"""FP64 CPU oracle for Guided Linear Upsampling (test infrastructure only).

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this package. It
shares no code with the CUDA library in paper_2307_09582_gb300.
"""
