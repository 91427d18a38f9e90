"""GB300-native (sm_103a) neural path tracer: the data-parallel hot path of
"Towards Neural Path Tracing in SRAM" (Pupilli 2023) behind a C ABI."""
