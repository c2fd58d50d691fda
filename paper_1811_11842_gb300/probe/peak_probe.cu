// Rate probe: FP64 and FP32 FMA throughput (8 independent FMA chains per
// thread, 152 x 8 blocks of 256 threads), streaming copy bandwidth and the
// back-to-back launch interval.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o peak_probe peak_probe.cu && ./peak_probe
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)
template<typename T> __global__ void fma_kernel(T* out, int iters, T a, T b){
  T x0=threadIdx.x*1e-3, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int k=0;k<iters;k++){
    x0=fma(x0,a,b); x1=fma(x1,a,b); x2=fma(x2,a,b); x3=fma(x3,a,b);
    x4=fma(x4,a,b); x5=fma(x5,a,b); x6=fma(x6,a,b); x7=fma(x7,a,b);
  }
  T s=x0+x1+x2+x3+x4+x5+x6+x7;
  if(s==(T)-1.2345) out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void copy_kernel(const double2* __restrict__ a, double2* __restrict__ b, size_t n){
  size_t i=blockIdx.x*(size_t)blockDim.x+threadIdx.x, st=(size_t)gridDim.x*blockDim.x;
  for(;i<n;i+=st) b[i]=a[i];
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  printf("name=%s sms=%d l2=%d smem_optin=%zu clock_khz=? \n",p.name,p.multiProcessorCount,p.l2CacheSize,p.sharedMemPerBlockOptin);
  int blocks=p.multiProcessorCount*8, threads=256;
  double* outd; float* outf; CK(cudaMalloc(&outd,blocks*threads*8)); CK(cudaMalloc(&outf,blocks*threads*4));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for(int rep=0;rep<3;rep++){
    int it=4096;
    fma_kernel<double><<<blocks,threads>>>(outd,16,1.0000001,1e-9);
    cudaEventRecord(e0); fma_kernel<double><<<blocks,threads>>>(outd,it,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*it*(double)blocks*threads; printf("fp64 fma: %.3f ms  %.1f GFLOP/s\n",ms,fl/ms/1e6);
    it=65536;
    cudaEventRecord(e0); fma_kernel<float><<<blocks,threads>>>(outf,it,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    fl=2.0*8*it*(double)blocks*threads; printf("fp32 fma: %.3f ms  %.1f GFLOP/s\n",ms,fl/ms/1e6);
  }
  size_t bytes=(size_t)1<<31; size_t n=bytes/16; double2 *a,*b; CK(cudaMalloc(&a,bytes)); CK(cudaMalloc(&b,bytes));
  CK(cudaMemset(a,0,bytes)); CK(cudaMemset(b,0,bytes));
  for(int rep=0;rep<5;rep++){
    cudaEventRecord(e0); copy_kernel<<<p.multiProcessorCount*16,512>>>(a,b,n); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("copy 2x%zu MB: %.3f ms %.1f GB/s\n",bytes>>20,ms,2.0*bytes/ms/1e6);
  }
  // small (L2-resident) copy: 16 MB
  size_t sb=16<<20; size_t sn=sb/16;
  for(int rep=0;rep<5;rep++){
    cudaEventRecord(e0); for(int k=0;k<20;k++) copy_kernel<<<p.multiProcessorCount*4,512>>>(a,b,sn); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("copy 16MB x20 (L2): %.3f ms/launch %.1f GB/s\n",ms/20,20*2.0*sb/ms/1e6);
  }
  // launch latency: empty-ish dependent launches
  cudaEventRecord(e0); for(int k=0;k<1000;k++) copy_kernel<<<152,256>>>(a,b,0); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&ms,e0,e1); printf("empty launch: %.2f us each\n",ms);
  CK(cudaGetLastError());
  return 0;
}
